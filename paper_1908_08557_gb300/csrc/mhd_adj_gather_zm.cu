// mhd_adj_gather_zm.cu -- the transposed-stencil gather of the adjoint right-
// hand side as a z-march.
//
// Given the 40 coefficient fields h of a substep (the adjoints of the cell
// values and of every derivative the right-hand side read, [q][nz][ny][nx]),
// the adjoint of the ghost-filled input is, per output field,
//   sum over first-derivative coefficients   D1_a^T h = -D1_a h,
//   + Laplacian coefficients                  (D2x + D2y + D2z) h,
//   + gradient-of-divergence coefficients     D2_a h (own axis) and
//                                             D1_a D1_c h (c != a, symmetric),
//   + value coefficients (u, ln rho, ln T),
// periodic in x and y, zero outside the interior layers, evaluated on the
// interior and the three z ghost layers on each side.
//
// A CTA (256 threads, one cell each) owns a 32 x 8 tile and one output group
// -- {A_x, A_y, A_z, ln rho} or {u_x, u_y, u_z, ln T}, 20 coefficient fields
// each -- and marches over the coefficient planes p of a z chunk.  Plane p of
// the group's 20 fields (with a 3-cell x, y halo, wrapped periodically) is
// staged in shared memory by cp.async in 16-byte chunks (one chunk position
// per thread, all 20 fields), double-buffered.  Items run tile-fastest, so
// CTAs working at the same time share z chunks and their halo planes in L2.  Its in-plane terms go
// to the output at plane p; the z terms are scattered from the cell's column:
// h(p) contributes to outputs p - 3 .. p + 3, held in a 7-plane accumulator
// ring per output field in registers.  When plane p is done, output plane
// p - 3 is complete and is written.  The in-plane mixed terms D1x D1y use the
// commuted form D1x(D1y h) through a scratch row with an x halo.
//
// Output (as in the 3D-tiled gather): on layers klo <= k < khi the substep's
// update F += G, D = alpha D + beta F; elsewhere G into gbar, with the value
// adjoints of the photospheric nudging (A_x, A_y at k = 0, Eq. 4) and of the
// stateful u_x, u_y ghost rows (Eq. 5).
#include "mhd_adjoint_point.cuh"
#include "mhd_internal.h"
#include "mhd_pair.cuh"
#include "mhd_zmarch.cuh"

namespace mhd {
namespace gzm {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int XO = 4;                 // staged rows start 4 columns left of the tile
constexpr int SX = TX + 8, SY = TY + 6;
constexpr int SP = SX * SY;           // elements of one staged field plane
constexpr int NQ = 20;                // coefficient fields of an output group
constexpr int NO = 4;                 // output fields of a group

template <typename R> constexpr size_t smem_bytes() {
  return (size_t)2 * NQ * SP * sizeof(R) + (size_t)4 * TY * SX * sizeof(R);
}

// staged order of the coefficient fields: 0..8 first derivatives (component
// c, axis a at 3c + a), 9..11 Laplacians, 12..14 gradient-of-divergence (A)
// or values (u), 15 value, 16..18 gradient, 19 Laplacian of the scalar
__constant__ int kQ[2][NQ] = {
    {CDA + 0, CDA + 1, CDA + 2, CDA + 3, CDA + 4, CDA + 5, CDA + 6, CDA + 7, CDA + 8, CLA + 0, CLA + 1, CLA + 2,
     CGA + 0, CGA + 1, CGA + 2, CV + LR, CGL + 0, CGL + 1, CGL + 2, CLL},
    {CDU + 0, CDU + 1, CDU + 2, CDU + 3, CDU + 4, CDU + 5, CDU + 6, CDU + 7, CDU + 8, CLU + 0, CLU + 1, CLU + 2,
     CV + UX, CV + UY, CV + UZ, CV + LT, CGT + 0, CGT + 1, CGT + 2, CLT}};

template <typename R>
struct ZArgs {
  Layout L;
  Phys<R> ph;
  const R* coef;
  R* dbar;
  R* gbar;
  R* fbar;
  R alpha, beta;
  int klo, khi;
  StepState* ss;
  int ntx, nty, nch, kchunk;
};

// stencils on a staged plane at offset c (stride s), unscaled
template <typename R> __device__ __forceinline__ R sd1(const R* p, int c, int s) {
  return W<R>::c1 * (p[c + s] - p[c - s]) + W<R>::c2 * (p[c + 2 * s] - p[c - 2 * s]) +
         W<R>::c3 * (p[c + 3 * s] - p[c - 3 * s]);
}
template <typename R> __device__ __forceinline__ R sd2(const R* p, int c, int s) {
  return W<R>::e0 * p[c] + W<R>::e1 * (p[c + s] + p[c - s]) + W<R>::e2 * (p[c + 2 * s] + p[c - 2 * s]) +
         W<R>::e3 * (p[c + 3 * s] + p[c - 3 * s]);
}

// z scatters into a 7-plane ring (index 3 = the current plane)
// D1z^T h:  +c_m h into p + m, -c_m h into p - m
template <typename R> __device__ __forceinline__ void z_d1t(R (&a)[7], R v) {
  a[4] += W<R>::c1 * v; a[2] -= W<R>::c1 * v;
  a[5] += W<R>::c2 * v; a[1] -= W<R>::c2 * v;
  a[6] += W<R>::c3 * v; a[0] -= W<R>::c3 * v;
}
// D1z f:  +c_m f into p - m, -c_m f into p + m
template <typename R> __device__ __forceinline__ void z_d1(R (&a)[7], R v) { z_d1t<R>(a, -v); }
// D2z h (symmetric)
template <typename R> __device__ __forceinline__ void z_d2(R (&a)[7], R v) {
  a[3] += W<R>::e0 * v;
  a[4] += W<R>::e1 * v; a[2] += W<R>::e1 * v;
  a[5] += W<R>::e2 * v; a[1] += W<R>::e2 * v;
  a[6] += W<R>::e3 * v; a[0] += W<R>::e3 * v;
}

template <typename R>
struct Smem {
  R* buf;          // [2][NQ][SP]
  R* scr;          // [2 buffers][2 fields][TY][SX]
};

// One item: output group GRP of a tile over output planes [n0, n1).
template <typename R, int GRP>
__device__ __forceinline__ void item_body(const ZArgs<R>& a, const Smem<R>& sm, int x0, int y0, int n0, int n1) {
  const Layout& L = a.L;
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long n2 = (long long)nx * ny, n3 = n2 * nz;
  const Phys<R>& ph = a.ph;
  const R idx = ph.idx, idy = ph.idy, idz = ph.idz, idx2 = ph.idx2, idy2 = ph.idy2, idz2 = ph.idz2;
  const R dt = R(a.ss->dt);
  const int cen = (ty + 3) * SX + tx + XO;
  const int pa = max(0, n0 - NG), pb = min(nz - 1, n1 + NG - 1);  // valid input planes
  // cp.async staging: thread tid copies 16-byte chunk position tid (and
  // tid + NT, if it exists) of the 20 field planes; source offsets within a
  // plane wrap periodically in x and y
  constexpr int EPC = 16 / (int)sizeof(R), CR = SX / EPC, CP = CR * SY;
  auto chunk_off = [&](int c) -> long long {
    if (c >= CP) return 0;
    const int r = c / CR, cc = c - r * CR;
    const int yy = ((y0 - 3 + r) % ny + ny) % ny, xx = ((x0 - XO + cc * EPC) % nx + nx) % nx;
    return (long long)yy * nx + xx;
  };
  const long long off0 = chunk_off(tid), off1 = chunk_off(tid + NT);
  auto cp16 = [](R* dst, const R* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(zm::sa(dst)), "l"(src) : "memory");
  };
  auto stage = [&](int p, int b) {
    R* dst = sm.buf + b * NQ * SP;
    const R* src = a.coef + (long long)p * n2;
    if (tid < CP) {
#pragma unroll 4
      for (int q = 0; q < NQ; ++q) cp16(dst + q * SP + tid * EPC, src + (long long)kQ[GRP][q] * n3 + off0);
    }
    if (tid + NT < CP) {
#pragma unroll 4
      for (int q = 0; q < NQ; ++q) cp16(dst + q * SP + (tid + NT) * EPC, src + (long long)kQ[GRP][q] * n3 + off1);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (pa <= pb) stage(pa, 0);
  int b = 0;
  R acc[NO][7];
#pragma unroll
  for (int t = 0; t < NO; ++t)
#pragma unroll
    for (int d = 0; d < 7; ++d) acc[t][d] = R(0);
  const int i = x0 + tx, j = y0 + ty;
  const bool live = i < nx && j < ny;
  // x-halo items of the in-plane mixed scratch: 2 fields x 8 rows x 6 columns
  const int hf = tid / 48, hr = (tid % 48) / 6, hcol = (tid % 6) < 3 ? 1 + tid % 6 : 33 + tid % 6;
  constexpr R g = GRP == 0 ? R(1) : R(1.0 / 3.0);

  for (int p = n0 - NG; p <= n1 + NG - 1; ++p) {
    // output plane p - 3 is written at the end of this plane: its
    // accumulator and D values are fetched now, ahead of the compute
    const int n = p - NG;
    const bool emit = n >= n0 && live;
    const bool fz = n >= a.klo && n < a.khi;
    R fo[NO], dd[NO];
#pragma unroll
    for (int t = 0; t < NO; ++t) {
      const int f = GRP == 0 ? (t < 3 ? AX + t : LR) : (t < 3 ? UX + t : LT);
      const long long q = emit ? L.at(f, n, j, i) : 0;
      fo[t] = (emit && fz) ? a.fbar[q] : R(0);
      dd[t] = (emit && (fz || (ph.bcz == 0 && n <= 0))) ? a.dbar[q] : R(0);
    }
    if (p >= pa && p <= pb) {
      if (p + 1 <= pb) {
        stage(p + 1, b ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const R* s = sm.buf + b * NQ * SP;
      auto S = [&](int q) { return s + q * SP; };
      // first derivatives of the three components: -D1x, -D1y, D1z^T
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[c][3] -= idx * sd1<R>(S(3 * c), cen, 1) + idy * sd1<R>(S(3 * c + 1), cen, SX);
        z_d1t<R>(acc[c], idz * S(3 * c + 2)[cen]);
      }
      // Laplacians (u: with the own-axis part of grad div u = lap u / 3)
      const R f43 = R(4.0 / 3.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R* h = S(9 + c);
        const R wx = (GRP == 1 && c == 0) ? f43 : R(1), wy = (GRP == 1 && c == 1) ? f43 : R(1);
        const R wz = (GRP == 1 && c == 2) ? f43 : R(1);
        acc[c][3] += wx * idx2 * sd2<R>(h, cen, 1) + wy * idy2 * sd2<R>(h, cen, SX);
        z_d2<R>(acc[c], wz * idz2 * h[cen]);
      }
      // gradient of divergence: gd_a coefficients (A: fields 12..14; u:
      // the Laplacian ones / 3)
      const R* gx = GRP == 0 ? S(12) : S(9);
      const R* gy = GRP == 0 ? S(13) : S(10);
      const R* gz = GRP == 0 ? S(14) : S(11);
      if (GRP == 0) {
        // own-axis parts (for u they are in the weighted Laplacians)
        acc[0][3] += idx2 * sd2<R>(gx, cen, 1);
        acc[1][3] += idy2 * sd2<R>(gy, cen, SX);
        z_d2<R>(acc[2], idz2 * gz[cen]);
      } else {
        // values of u
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c][3] += S(12 + c)[cen];
      }
      // xz, yz, zx, zy mixed: D1z of in-plane first derivatives
      z_d1<R>(acc[2], g * idz * (idx * sd1<R>(gx, cen, 1) + idy * sd1<R>(gy, cen, SX)));
      z_d1<R>(acc[0], g * idz * idx * sd1<R>(gz, cen, 1));
      z_d1<R>(acc[1], g * idz * idy * sd1<R>(gz, cen, SX));
      // xy mixed: D1x(D1y gd_x) -> component y, D1x(D1y gd_y) -> component x
      // (scratch double-buffered like the staged planes: a thread writes
      // buffer b only after every thread has passed the previous barrier)
      R* scr = sm.scr + b * 2 * TY * SX;
      scr[ty * SX + tx + XO] = sd1<R>(gx, cen, SX);
      scr[TY * SX + ty * SX + tx + XO] = sd1<R>(gy, cen, SX);
      if (tid < 96) scr[hf * TY * SX + hr * SX + hcol] = sd1<R>(hf == 0 ? gx : gy, (hr + 3) * SX + hcol, SX);
      // the scalar: value, -D1x, -D1y, D1z^T, Laplacian
      acc[3][3] += S(15)[cen] - idx * sd1<R>(S(16), cen, 1) - idy * sd1<R>(S(17), cen, SX) +
                   idx2 * sd2<R>(S(19), cen, 1) + idy2 * sd2<R>(S(19), cen, SX);
      z_d1t<R>(acc[3], idz * S(18)[cen]);
      z_d2<R>(acc[3], idz2 * S(19)[cen]);
      // every thread is done with staged buffer b and scratch b is complete
      __syncthreads();
      {
        const int o = ty * SX + tx + XO;
        acc[1][3] += g * idx * idy * sd1<R>(scr, o, 1);
        acc[0][3] += g * idx * idy * sd1<R>(scr + TY * SX, o, 1);
      }
      b ^= 1;
    }
    // output plane p - 3 is complete
    if (emit) {
#pragma unroll
      for (int t = 0; t < NO; ++t) {
        const int f = GRP == 0 ? (t < 3 ? AX + t : LR) : (t < 3 ? UX + t : LT);
        const long long q = L.at(f, n, j, i);
        const R v = acc[t][0];
        if (fz) {
          const R fv = fo[t] + v;
          a.fbar[q] = fv;
          a.dbar[q] = a.alpha * dd[t] + a.beta * fv;
        } else {
          R gv = v;
          if (ph.bcz == 0 && ((n == 0 && (f == AX || f == AY)) || (n < 0 && (f == UX || f == UY))))
            gv -= (f == AX || f == AY ? ph.tau_A : ph.tau_u) * dt * dd[t];
          a.gbar[q] = gv;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NO; ++t) {
#pragma unroll
      for (int d = 0; d < 6; ++d) acc[t][d] = acc[t][d + 1];
      acc[t][6] = R(0);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) gather_zm_kernel(ZArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<R> sm;
  sm.buf = reinterpret_cast<R*>(smem_raw);
  sm.scr = sm.buf + 2 * NQ * SP;
  if (halted(a.ss)) return;
  const int nzo = a.L.nz + 2 * NG;  // output planes -3 .. nz + 2
  const int nitems = a.ntx * a.nty * a.nch * 2;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int grp = item & 1;
    const int rest = item >> 1;
    const int tiles = a.ntx * a.nty;
    const int ch = rest / tiles, tile = rest % tiles;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int n0 = ch * a.kchunk - NG, n1 = min(nzo, (ch + 1) * a.kchunk) - NG;  // output planes [n0, n1)
    __syncthreads();  // the previous item's readers are done with the buffers
    if (grp == 0)
      item_body<R, 0>(a, sm, x0, y0, n0, n1);
    else
      item_body<R, 1>(a, sm, x0, y0, n0, n1);
  }
}

// ---------------------------------------------------------------------------
// FP32: the same z-march with two x-adjacent cells per thread in packed f32x2
// arithmetic (128 threads per 32 x 8 tile; 8-byte shared loads and global
// accesses).  The x stencils assemble the odd-offset pairs from even ones.
namespace zp {
using namespace pk;
constexpr int NTP = TX / 2 * TY;  // 128 threads
constexpr int CP = SX / 4 * SY;   // 16-byte chunks of a staged field plane (140)

__device__ __forceinline__ void zs_d1t(f2 (&a)[7], f2 v) {  // D1z^T
  a[4] = fma2(F2(W<float>::c1), v, a[4]); a[2] = fma2(F2(-W<float>::c1), v, a[2]);
  a[5] = fma2(F2(W<float>::c2), v, a[5]); a[1] = fma2(F2(-W<float>::c2), v, a[1]);
  a[6] = fma2(F2(W<float>::c3), v, a[6]); a[0] = fma2(F2(-W<float>::c3), v, a[0]);
}
__device__ __forceinline__ void zs_d1(f2 (&a)[7], f2 v) {  // D1z
  a[2] = fma2(F2(W<float>::c1), v, a[2]); a[4] = fma2(F2(-W<float>::c1), v, a[4]);
  a[1] = fma2(F2(W<float>::c2), v, a[1]); a[5] = fma2(F2(-W<float>::c2), v, a[5]);
  a[0] = fma2(F2(W<float>::c3), v, a[0]); a[6] = fma2(F2(-W<float>::c3), v, a[6]);
}
__device__ __forceinline__ void zs_d2(f2 (&a)[7], f2 v) {  // D2z
  a[3] = fma2(F2(W<float>::e0), v, a[3]);
  a[4] = fma2(F2(W<float>::e1), v, a[4]); a[2] = fma2(F2(W<float>::e1), v, a[2]);
  a[5] = fma2(F2(W<float>::e2), v, a[5]); a[1] = fma2(F2(W<float>::e2), v, a[1]);
  a[6] = fma2(F2(W<float>::e3), v, a[6]); a[0] = fma2(F2(W<float>::e3), v, a[0]);
}
// second derivative only
__device__ __forceinline__ f2 dxx(const float* p, const Coef& c) {
  f2 d1, d2;
  dx_pair(p, c, d1, &d2);
  return d2;
}
__device__ __forceinline__ f2 dyy(const float* p, const Coef& c) {
  f2 d1, d2;
  ds_pair(p, SX, c, d1, &d2);
  return d2;
}
__device__ __forceinline__ f2 dx1(const float* p, const Coef& c) {
  f2 d1;
  dx_pair(p, c, d1, nullptr);
  return d1;
}
__device__ __forceinline__ f2 dy1(const float* p, const Coef& c) {
  f2 d1;
  ds_pair(p, SX, c, d1, nullptr);
  return d1;
}

struct PArgs {
  ZArgs<float> z;
  Coef cx, cy;  // D1, D2 weights over dx, dy
  int dyn;      // items claimed from the step state's counter (else grid stride)
};

// Staged fields.  Only the coefficients whose in-plane stencils the gather
// takes need the x, y halo in shared memory; the ones it reads at the cell
// alone (the z-derivative coefficients, the values) are loaded straight from
// global memory, as 8-byte pairs of the thread's two cells.  Staged slot of
// the group's field q (-1: read at the cell), and the centre slot (-1: staged).
constexpr int NHP = 15;   // staged fields, at most (group 0; group 1 stages 12)
constexpr int NCP = 8;    // centre-only fields, at most (group 1; group 0 reads 5)
constexpr int NBP = 3;    // plane buffers: two planes in flight while one is used
__host__ __device__ constexpr int hslot(int grp, int q) {
  return grp == 0 ? (q == 2 || q == 5 || q == 8 || q == 15 || q == 18
                         ? -1
                         : q < 2 ? q : q < 5 ? q - 1 : q < 8 ? q - 2 : q < 15 ? q - 3 : q < 18 ? q - 4 : q - 5)
                  : (q == 2 || q == 5 || q == 8 || (q >= 12 && q <= 15) || q == 18
                         ? -1
                         : q < 2 ? q : q < 5 ? q - 1 : q < 8 ? q - 2 : q < 12 ? q - 3 : q < 18 ? q - 7 : q - 8);
}
__host__ __device__ constexpr int cslot(int grp, int q) {
  return grp == 0 ? (q == 2 ? 0 : q == 5 ? 1 : q == 8 ? 2 : q == 15 ? 3 : q == 18 ? 4 : -1)
                  : (q == 2 ? 0 : q == 5 ? 1 : q == 8 ? 2 : (q >= 12 && q <= 15) ? q - 9 : q == 18 ? 7 : -1);
}
static_assert(hslot(0, 19) == 14 && hslot(1, 19) == 11 && hslot(1, 16) == 9 && cslot(1, 15) == 6, "slot maps");
constexpr size_t smem_pair() { return (size_t)NBP * NHP * SP * 4 + (size_t)4 * TY * SX * 4; }

template <int GRP>
__device__ __forceinline__ void item_pair(const PArgs& pa_, float* buf, float* scrb, int x0, int y0, int n0,
                                          int n1) {
  const ZArgs<float>& a = pa_.z;
  const Layout& L = a.L;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long n2 = (long long)nx * ny, n3 = n2 * nz;
  const Phys<float>& ph = a.ph;
  const float idz = ph.idz, idz2 = ph.idz2;
  const float dt = (float)a.ss->dt;
  const int e = 2 * tx + XO;
  const int cen = (ty + 3) * SX + e;
  const int pa = max(0, n0 - NG), pb = min(nz - 1, n1 + NG - 1);
  auto chunk_off = [&](int c) -> long long {
    if (c >= CP) return 0;
    const int r = c / (SX / 4), cc = c - r * (SX / 4);
    const int yy = ((y0 - 3 + r) % ny + ny) % ny, xx = ((x0 - XO + cc * 4) % nx + nx) % nx;
    return (long long)yy * nx + xx;
  };
  const long long off0 = chunk_off(tid), off1 = chunk_off(tid + NTP);
  auto cp16 = [](float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(zm::sa(dst)), "l"(src) : "memory");
  };
  auto stage = [&](int p, int bb) {
    float* dst = buf + bb * NHP * SP;
    const float* src = a.coef + (long long)p * n2;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int hs = hslot(GRP, q);
      if (hs < 0) continue;
      const long long fo = (long long)kQ[GRP][q] * n3;
      cp16(dst + hs * SP + tid * 4, src + fo + off0);
      if (tid + NTP < CP) cp16(dst + hs * SP + (tid + NTP) * 4, src + fo + off1);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (pa <= pb) stage(pa, 0);
  if (pa + 1 <= pb) stage(pa + 1, 1);
  int b = 0;
  f2 acc[NO][7];
#pragma unroll
  for (int t = 0; t < NO; ++t)
#pragma unroll
    for (int d = 0; d < 7; ++d) acc[t][d] = F2(0.f);
  const int i = x0 + 2 * tx, j = y0 + ty;
  const bool live = i < nx && j < ny;
  // x-halo pairs of the in-plane mixed scratch: 2 fields x 8 rows x 4 pairs
  const int hf = tid >> 5, hr = (tid & 31) >> 2, hx = (tid & 3) < 2 ? 2 * (tid & 3) : 32 + 2 * (tid & 3);
  const float g = GRP == 0 ? 1.f : 1.f / 3.f;
  const Coef& cx = pa_.cx;
  const Coef& cy = pa_.cy;
  const long long qc = (long long)j * nx + i;  // the pair's offset within a plane

  for (int p = n0 - NG; p <= n1 + NG - 1; ++p) {
    const int n = p - NG;
    const bool emit = n >= n0 && live;
    const bool fz = n >= a.klo && n < a.khi;
    f2 fo[NO], dd[NO];
    long long qo = 0;
    if (emit) qo = L.at(0, n, j, i);
#pragma unroll
    for (int t = 0; t < NO; ++t) {
      const int f = GRP == 0 ? (t < 3 ? AX + t : LR) : (t < 3 ? UX + t : LT);
      const long long q = qo + (long long)f * L.fs;
      fo[t] = (emit && fz) ? ld2(a.fbar + q) : F2(0.f);
      dd[t] = (emit && (fz || (ph.bcz == 0 && n <= 0))) ? ld2(a.dbar + q) : F2(0.f);
    }
    if (p >= pa && p <= pb) {
      // the centre-only coefficients of plane p (issued before the wait)
      f2 cv[NCP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int cs = cslot(GRP, q);
        if (cs < 0) continue;
        cv[cs] = live ? __ldg(reinterpret_cast<const float2*>(a.coef + (long long)kQ[GRP][q] * n3 + (long long)p * n2 + qc))
                      : F2(0.f);
      }
      if (p + 2 <= pb) {
        stage(p + 2, b == 0 ? 2 : b - 1);
        asm volatile("cp.async.wait_group 2;" ::: "memory");
      } else if (p + 1 <= pb) {
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const float* s = buf + b * NHP * SP;
      auto S = [&](int q) { return s + hslot(GRP, q) * SP + cen; };
      auto C = [&](int q) { return cv[cslot(GRP, q)]; };
      // first derivatives of the three components: -D1x, -D1y, D1z^T
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[c][3] = dif(acc[c][3], add(dx1(S(3 * c), cx), dy1(S(3 * c + 1), cy)));
        zs_d1t(acc[c], mul(F2(idz), C(3 * c + 2)));
      }
      // Laplacians (u: with the own-axis part of grad div u = lap u / 3)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* h = S(9 + c);
        const float wx = (GRP == 1 && c == 0) ? 4.f / 3.f : 1.f, wy = (GRP == 1 && c == 1) ? 4.f / 3.f : 1.f;
        const float wz = (GRP == 1 && c == 2) ? 4.f / 3.f : 1.f;
        acc[c][3] = fma2(F2(wx), dxx(h, cx), fma2(F2(wy), dyy(h, cy), acc[c][3]));
        zs_d2(acc[c], mul(F2(wz * idz2), ld2(h)));
      }
      const float* gx = GRP == 0 ? S(12) : S(9);
      const float* gy = GRP == 0 ? S(13) : S(10);
      const float* gz = GRP == 0 ? S(14) : S(11);
      if (GRP == 0) {
        acc[0][3] = add(acc[0][3], dxx(gx, cx));
        acc[1][3] = add(acc[1][3], dyy(gy, cy));
        zs_d2(acc[2], mul(F2(idz2), ld2(gz)));
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c][3] = add(acc[c][3], C(12 + c));
      }
      // xz, yz, zx, zy mixed: D1z of in-plane first derivatives
      const f2 gyy = dy1(gy, cy);
      zs_d1(acc[2], mul(F2(g * idz), add(dx1(gx, cx), gyy)));
      zs_d1(acc[0], mul(F2(g * idz), dx1(gz, cx)));
      zs_d1(acc[1], mul(F2(g * idz), dy1(gz, cy)));
      // xy mixed through the x-halo scratch: D1x(D1y gd_x) -> y, D1x(D1y gd_y) -> x
      float* scr = scrb + ((p - pa) & 1) * 2 * TY * SX;
      *reinterpret_cast<f2*>(scr + ty * SX + e) = dy1(gx, cy);
      *reinterpret_cast<f2*>(scr + TY * SX + ty * SX + e) = gyy;
      if (tid < 64)
        *reinterpret_cast<f2*>(scr + hf * TY * SX + hr * SX + hx) =
            dy1(s + hslot(GRP, GRP == 0 ? 12 + hf : 9 + hf) * SP + (hr + 3) * SX + hx, cy);
      // the scalar: value, -D1x, -D1y, D1z^T, Laplacian
      acc[3][3] = add(acc[3][3], dif(add(C(15), add(dxx(S(19), cx), dyy(S(19), cy))),
                                     add(dx1(S(16), cx), dy1(S(17), cy))));
      zs_d1t(acc[3], mul(F2(idz), C(18)));
      zs_d2(acc[3], mul(F2(idz2), ld2(S(19))));
      __syncthreads();
      acc[1][3] = fma2(F2(g), dx1(scr + ty * SX + e, cx), acc[1][3]);
      acc[0][3] = fma2(F2(g), dx1(scr + TY * SX + ty * SX + e, cx), acc[0][3]);
      b = b == NBP - 1 ? 0 : b + 1;
    }
    if (emit) {
#pragma unroll
      for (int t = 0; t < NO; ++t) {
        const int f = GRP == 0 ? (t < 3 ? AX + t : LR) : (t < 3 ? UX + t : LT);
        const long long q = qo + (long long)f * L.fs;
        const f2 v = acc[t][0];
        if (fz) {
          const f2 fv = add(fo[t], v);
          *reinterpret_cast<f2*>(a.fbar + q) = fv;
          *reinterpret_cast<f2*>(a.dbar + q) = fma2(F2(a.alpha), dd[t], mul(F2(a.beta), fv));
        } else {
          f2 gv = v;
          if (ph.bcz == 0 && ((n == 0 && (f == AX || f == AY)) || (n < 0 && (f == UX || f == UY))))
            gv = dif(gv, mul(F2((f == AX || f == AY ? ph.tau_A : ph.tau_u) * dt), dd[t]));
          *reinterpret_cast<f2*>(a.gbar + q) = gv;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NO; ++t) {
#pragma unroll
      for (int d = 0; d < 6; ++d) acc[t][d] = acc[t][d + 1];
      acc[t][6] = F2(0.f);
    }
  }
}

__global__ void __launch_bounds__(NTP, 2) gather_pair_kernel(PArgs pa_) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  float* scr = buf + NBP * NHP * SP;
  const ZArgs<float>& a = pa_.z;
  if (halted(a.ss)) return;
  const int nzo = a.L.nz + 2 * NG;
  const int tiles = a.ntx * a.nty;
  const int nitems = tiles * a.nch * 2;
  // items group-major within a z chunk: the CTAs running together hold all
  // tiles of one output group, whose halo planes they share in L2.  With
  // several items per CTA (dyn) each CTA claims its next item from the step
  // state's counter as it starts one (the claim is handed to the CTA at the
  // end-of-item barrier), so that CTAs meeting dearer items (the x, y edges'
  // wrapped halos, the update layers) do not hold up the launch.
  __shared__ int s_next;
  if (pa_.dyn) {
    if (threadIdx.x == 0) s_next = atomicAdd(&a.ss->items, 1);
    __syncthreads();
  }
  for (int item = pa_.dyn ? s_next : (int)blockIdx.x; item < nitems;) {
    int next = 0;
    if (pa_.dyn && threadIdx.x == 0) next = atomicAdd(&a.ss->items, 1);
    const int ch = item / (2 * tiles), r = item - ch * 2 * tiles;
    const int grp = r >= tiles ? 1 : 0;
    const int tile = r - grp * tiles;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int n0 = ch * a.kchunk - NG, n1 = min(nzo, (ch + 1) * a.kchunk) - NG;
    __syncthreads();
    if (grp == 0)
      item_pair<0>(pa_, buf, scr, x0, y0, n0, n1);
    else
      item_pair<1>(pa_, buf, scr, x0, y0, n0, n1);
    if (pa_.dyn) {
      __syncthreads();
      if (threadIdx.x == 0) s_next = next;
      __syncthreads();
      item = s_next;
    } else {
      item += gridDim.x;
    }
  }
}
}  // namespace zp

}  // namespace gzm

template <typename R>
void launch_adj_gather_zm(const Layout& L, const Phys<R>& ph, const R* coef, R* dbar, R* gbar, R* fbar,
                          double alpha, double beta, int klo, int khi, StepState* ss, cudaStream_t st) {
  constexpr size_t smem = gzm::smem_bytes<R>();
  // persistent CTAs on the current device (shared-memory limit set there)
  static PerDevice<int> per_dev;
  const int ctas = per_dev.get([] {
    cudaFuncSetAttribute(gzm::gather_zm_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gzm::gather_zm_kernel<R>, gzm::NT, smem);
    return sm_count() * (per > 0 ? per : 1);
  });
  gzm::ZArgs<R> a;
  a.L = L;
  a.ph = ph;
  a.coef = coef;
  a.dbar = dbar;
  a.gbar = gbar;
  a.fbar = fbar;
  a.alpha = (R)alpha;
  a.beta = (R)beta;
  a.klo = klo;
  a.khi = khi;
  a.ss = ss;
  a.ntx = (L.nx + gzm::TX - 1) / gzm::TX;
  a.nty = (L.ny + gzm::TY - 1) / gzm::TY;
  const int tiles = a.ntx * a.nty;
  a.kchunk = zm::zchunk(L.nz + 2 * NG, 2 * tiles, ctas);
  a.nch = (L.nz + 2 * NG + a.kchunk - 1) / a.kchunk;
  const int nitems = 2 * tiles * a.nch;
  if constexpr (sizeof(R) == 4) {
    constexpr size_t psmem = gzm::zp::smem_pair();
    static PerDevice<int> per_dev_pair;
    const int pctas = per_dev_pair.get([] {
      cudaFuncSetAttribute(gzm::zp::gather_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gzm::zp::gather_pair_kernel, gzm::zp::NTP, psmem);
      return sm_count() * (per > 0 ? per : 1);
    });
    gzm::zp::PArgs pa;
    pa.z = a;
    a.kchunk = zm::zchunk(L.nz + 2 * NG, 2 * tiles, pctas);
    a.nch = (L.nz + 2 * NG + a.kchunk - 1) / a.kchunk;
    pa.z = a;
    const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
    const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0, 2.0 / 180.0};
    auto coef = [&](double h) {
      pk::Coef c;
      c.c1 = pk::F2((float)(W1[1] / h)); c.c2 = pk::F2((float)(W1[2] / h)); c.c3 = pk::F2((float)(W1[3] / h));
      c.e0 = pk::F2((float)(W2[0] / (h * h))); c.e1 = pk::F2((float)(W2[1] / (h * h)));
      c.e2 = pk::F2((float)(W2[2] / (h * h))); c.e3 = pk::F2((float)(W2[3] / (h * h)));
      return c;
    };
    pa.cx = coef(1.0 / (double)ph.idx);
    pa.cy = coef(1.0 / (double)ph.idy);
    const int pitems = 2 * tiles * a.nch;
    const int pgrid = pitems < pctas ? pitems : pctas;
    pa.dyn = pitems >= 4 * pgrid;
    if (pa.dyn) cudaMemsetAsync(&ss->items, 0, sizeof(int), st);
    gzm::zp::gather_pair_kernel<<<pgrid, gzm::zp::NTP, psmem, st>>>(pa);
    return;
  }
  gzm::gather_zm_kernel<R><<<nitems < ctas ? nitems : ctas, gzm::NT, smem, st>>>(a);
}

template void launch_adj_gather_zm<float>(const Layout&, const Phys<float>&, const float*, float*, float*, float*,
                                          double, double, int, int, StepState*, cudaStream_t);
template void launch_adj_gather_zm<double>(const Layout&, const Phys<double>&, const double*, double*, double*,
                                           double*, double, double, int, int, StepState*, cudaStream_t);

}  // namespace mhd
