// mhd_rk_split.cu -- FP32 right-hand side + RK3 update as two TMA-fed
// z-march passes, each small enough in shared memory for two CTAs per SM
// (the fused kernel's 8-field ring allows one):
//  pass A: stencils of A (3 fields) -> B = curl A + B_ext, J = grad div A -
//          lap A (Eq. 6) and the swamp terms of the induction equation, per
//          interior cell, into a compact buffer;
//  pass R: stencils of u, ln rho, ln T (5 fields), with A, B, J and the
//          swamp terms read per cell: the pointwise physics (rhs_point_bj),
//          boundary rows and nudging, the low-storage RK update and the
//          stores (with periodic images).
// As in the fused kernel a CTA owns a 32 x 8 tile and marches in z; plane p
// of its fields arrives through one 4D cp.async.bulk.tensor load into an
// 8-slot ring guarded by mbarriers (bounded waits).  The z histories of the
// mixed-derivative sources (D1x X_z, D1y X_z, D1x X_x + D1y X_y over planes
// k-3 .. k+3) and of the xy-mixed terms (planes k .. k+3) are kept in each
// thread's registers: a thread keeps its (x, y) column for the whole chunk.
#include "mhd_internal.h"
#include "mhd_zmarch.cuh"

namespace mhd {
namespace split {

using zm::BX;
using zm::BY;
using zm::FItems;
using zm::TILE;
using zm::TX;
using zm::TY;
using zm::WXH;
using zm::WYW;
using zm::D1;
using zm::D2;

constexpr int NRAW = 8;              // raw ring: planes k-3 .. k+4
constexpr int NFA = 3, NFR = 5;      // fields per plane: pass A (A), pass R (u, ln rho, ln T)
constexpr int PA = NFA * BY * BX, PR = NFR * BY * BX;  // floats per box plane
// ring slots start on 128-byte boundaries (TMA destination alignment)
constexpr int slot_floats(int plane) { return (plane + 31) / 32 * 32; }
constexpr int SA = slot_floats(PA), SR = slot_floats(PR);
constexpr size_t smem_bytes(int slot) {
  return (size_t)NRAW * slot * 4 + (size_t)(TY * WYW + WXH * TX) * 4 + NRAW * 8;
}
constexpr size_t SMEM_A = smem_bytes(SA);
constexpr size_t SMEM_R = smem_bytes(SR);

struct Args {
  Layout L;
  Phys<float> ph;
  Background<float> bg;
  const float* fin;   // input state (pass R reads A at the cell)
  float* fout;
  float* df;
  float* bj;          // [6][nz][ny][nx]: B, J
  float* sw;          // [3][nz - ksw][ny][nx]: swamp terms of the layers k >= ksw
  int ksw;
  const float* wtab;
  const float* wptab;
  const float* axt;
  const float* ayt;
  const float* v0;
  const float* v1;
  StepState* ss;
  int sub;
  int ntx, nty, nch, kchunk;
  float c1x, c2x, c3x, c1y, c2y, c3y, c1z, c2z, c3z;
  float e0x, e1x, e2x, e3x, e0y, e1y, e2y, e3y, e0z, e1z, e2z, e3z;
};

// Ring bookkeeping shared by both passes: a tile/chunk work item, the
// initial TMA loads, the bounded wait for a plane, the refill after a centre
// plane, and the drain after a time-out.
struct Ring {
  uint64_t* mbar;
  uint32_t phase = 0;    // bit s: parity of the next completion of slot s
  uint32_t pending = 0;  // bit s: a copy into slot s is in flight
  __device__ void init(int tid) {
    if (tid == 0) {
      for (int s = 0; s < NRAW; ++s) zm::mbar_init(&mbar[s]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
  }
  __device__ void load(const CUtensorMap* tm, float* raw, int stride, unsigned bytes, int slot, int x0, int y0,
                       int p, int f0) {
    zm::tma_plane(tm, raw + slot * stride, &mbar[slot], bytes, x0 - 4 + XOFF, y0, p + NG, f0);
    pending |= 1u << slot;
  }
  // collective: false (for every thread) if any thread's wait timed out
  __device__ bool wait(int slot) {
    const bool to = !zm::mbar_wait(&mbar[slot], (phase >> slot) & 1u);
    if (__syncthreads_or(to)) return false;
    phase ^= 1u << slot;
    pending &= ~(1u << slot);
    return true;
  }
  __device__ void drain(int tid, StepState* ss) {
    if (tid == 0) {
      atomicOr(&ss->nonfinite, 2);
      for (int s = 0; s < NRAW; ++s)
        if (pending & (1u << s)) zm::mbar_wait(&mbar[s], (phase >> s) & 1u);
    }
  }
};

// register z histories: d[q][m] = source q of plane k-3+m (m = 0..6),
// mx[q][m] = xy-mixed term q of plane k+m (m = 0..3), after the front of k+3
struct Hist {
  float d[3][7];
  float mx[2][4];
  __device__ __forceinline__ void push(float d0, float d1, float d2, float m0, float m1) {
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      d[0][m] = d[0][m + 1];
      d[1][m] = d[1][m + 1];
      d[2][m] = d[2][m + 1];
    }
    d[0][6] = d0;
    d[1][6] = d1;
    d[2][6] = d2;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      mx[0][m] = mx[0][m + 1];
      mx[1][m] = mx[1][m + 1];
    }
    mx[0][3] = m0;
    mx[1][3] = m1;
  }
  // D1z of source q at the centre
  __device__ __forceinline__ float dz(int q, float c1, float c2, float c3) const {
    return c1 * (d[q][4] - d[q][2]) + c2 * (d[q][5] - d[q][1]) + c3 * (d[q][6] - d[q][0]);
  }
};

// Front processing of plane P (fields of one vector X at offsets fx, fy, fz
// inside the box plane): D1x X_z, D1y X_z at the cell; D1y X_y on the tile
// plus x halo and D1x X_x on the tile plus y halo through shared memory, then
// D1x(D1y X_y), D1y(D1x X_x) and D1x X_x + D1y X_y at the cell.
__device__ __forceinline__ void front(const Args& a, const FItems& it, const float* __restrict__ P, int fx, int fy,
                                      int fz, float* __restrict__ wy, float* __restrict__ wx, int cen, int tx,
                                      int ty, Hist& h) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < it.n) {
      if (it.isy[t])
        wy[it.dst[t]] = D1(P + fy * BY * BX + it.src[t], BX, a.c1y, a.c2y, a.c3y);
      else
        wx[it.dst[t]] = D1(P + fx * BY * BX + it.src[t], 1, a.c1x, a.c2x, a.c3x);
    }
  }
  const float d0 = D1(P + fz * BY * BX + cen, 1, a.c1x, a.c2x, a.c3x);
  const float d1 = D1(P + fz * BY * BX + cen, BX, a.c1y, a.c2y, a.c3y);
  __syncthreads();
  const float* wyc = wy + ty * WYW + tx + 3;
  const float* wxc = wx + (ty + 3) * TX + tx;
  const float m0 = D1(wyc, 1, a.c1x, a.c2x, a.c3x);
  const float m1 = D1(wxc, TX, a.c1y, a.c2y, a.c3y);
  const float d2 = wxc[0] + wyc[0];
  __syncthreads();
  h.push(d0, d1, d2, m0, m1);
}

// values, first and second derivatives of field f of the ring at the centre
struct Deriv {
  float v, dx, dy, dz, xx, yy, zz;
};
__device__ __forceinline__ Deriv deriv(const Args& a, const float* const (&Pz)[7], int f) {
  const int o = f * BY * BX;
  const float* p = Pz[3] + o;
  Deriv d;
  d.v = p[0];
  d.dx = D1(p, 1, a.c1x, a.c2x, a.c3x);
  d.dy = D1(p, BX, a.c1y, a.c2y, a.c3y);
  d.xx = D2(p, 1, a.e0x, a.e1x, a.e2x, a.e3x);
  d.yy = D2(p, BX, a.e0y, a.e1y, a.e2y, a.e3y);
  d.dz = a.c1z * (Pz[4][o] - Pz[2][o]) + a.c2z * (Pz[5][o] - Pz[1][o]) + a.c3z * (Pz[6][o] - Pz[0][o]);
  d.zz = a.e0z * Pz[3][o] + a.e1z * (Pz[4][o] + Pz[2][o]) + a.e2z * (Pz[5][o] + Pz[1][o]) +
         a.e3z * (Pz[6][o] + Pz[0][o]);
  return d;
}

// ---------------------------------------------------------------------------
// pass A
__global__ void __launch_bounds__(TILE, 3) pass_a_kernel(const __grid_constant__ CUtensorMap tm, const Args a) {
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;
  float* wy = raw + NRAW * SA;
  float* wx = wy + TY * WYW;
  Ring ring;
  ring.mbar = (uint64_t*)(wx + WXH * TX);
  const Layout& L = a.L;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  if (halted(a.ss)) return;
  ring.init(tid);
  const FItems items = zm::make_items(tid);
  const int cen = (ty + 3) * BX + tx + 4;
  const int nitems = a.ntx * a.nty * a.nch;
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  bool bad = false;
  Hist h = {};

  for (int item = blockIdx.x; item < nitems && !bad; item += gridDim.x) {
    const int ch = item % a.nch, tile = item / a.nch;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int k0 = ch * a.kchunk, k1 = min(L.nz, k0 + a.kchunk);
    const int pbase = k0 - NG, plast = k1 + NG - 1;
    if (tid == 0)
      for (int p = pbase; p <= min(pbase + NRAW - 1, plast); ++p)
        ring.load(&tm, raw, SA, PA * 4, (p - pbase) & (NRAW - 1), x0, y0, p, AX);
    for (int p = pbase; p < k0 + NG && !bad; ++p) {
      const int s = (p - pbase) & (NRAW - 1);
      bad = !ring.wait(s);
      if (!bad) front(a, items, raw + s * SA, AX, AY, AZ, wy, wx, cen, tx, ty, h);
    }
    for (int k = k0; k < k1 && !bad; ++k) {
      {
        const int s = (k + NG - pbase) & (NRAW - 1);
        bad = !ring.wait(s);
        if (bad) break;
        front(a, items, raw + s * SA, AX, AY, AZ, wy, wx, cen, tx, ty, h);
      }
      const int i = x0 + tx, j = y0 + ty;
      if (i < L.nx && j < L.ny) {
        const int kr = k - pbase;
        const float* Pz[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) Pz[m] = raw + ((kr - 3 + m) & (NRAW - 1)) * SA + cen;
        float B[3], J[3], sw[3] = {0.f, 0.f, 0.f};
        const float dzx = h.dz(0, a.c1z, a.c2z, a.c3z);  // D1z D1x A_z
        const float dzy = h.dz(1, a.c1z, a.c2z, a.c3z);  // D1z D1y A_z
        const float dzd = h.dz(2, a.c1z, a.c2z, a.c3z);  // D1z (D1x A_x + D1y A_y)
        if (k < a.ksw) {
          // J = grad div A - lap A with each component's own-axis second
          // derivative cancelled (the same stencil appears in both terms);
          // the diagonal first derivatives only enter div A (swamp layers)
          const int ox = 0 * BY * BX, oy = 1 * BY * BX, oz = 2 * BY * BX;
          const float* px = Pz[3] + ox;
          const float* py = Pz[3] + oy;
          const float* pz = Pz[3] + oz;
          const float dyAx = D1(px, BX, a.c1y, a.c2y, a.c3y);
          const float dxAy = D1(py, 1, a.c1x, a.c2x, a.c3x);
          const float dxAz = D1(pz, 1, a.c1x, a.c2x, a.c3x);
          const float dyAz = D1(pz, BX, a.c1y, a.c2y, a.c3y);
          const float dzAx = a.c1z * (Pz[4][ox] - Pz[2][ox]) + a.c2z * (Pz[5][ox] - Pz[1][ox]) +
                             a.c3z * (Pz[6][ox] - Pz[0][ox]);
          const float dzAy = a.c1z * (Pz[4][oy] - Pz[2][oy]) + a.c2z * (Pz[5][oy] - Pz[1][oy]) +
                             a.c3z * (Pz[6][oy] - Pz[0][oy]);
          const float yyAx = D2(px, BX, a.e0y, a.e1y, a.e2y, a.e3y);
          const float xxAy = D2(py, 1, a.e0x, a.e1x, a.e2x, a.e3x);
          const float xxAz = D2(pz, 1, a.e0x, a.e1x, a.e2x, a.e3x);
          const float yyAz = D2(pz, BX, a.e0y, a.e1y, a.e2y, a.e3y);
          const float zzAx = a.e0z * Pz[3][ox] + a.e1z * (Pz[4][ox] + Pz[2][ox]) + a.e2z * (Pz[5][ox] + Pz[1][ox]) +
                             a.e3z * (Pz[6][ox] + Pz[0][ox]);
          const float zzAy = a.e0z * Pz[3][oy] + a.e1z * (Pz[4][oy] + Pz[2][oy]) + a.e2z * (Pz[5][oy] + Pz[1][oy]) +
                             a.e3z * (Pz[6][oy] + Pz[0][oy]);
          B[0] = dyAz - dzAy + a.ph.bext[0];
          B[1] = dzAx - dxAz + a.ph.bext[1];
          B[2] = dxAy - dyAx + a.ph.bext[2];
          J[0] = h.mx[0][0] + dzx - yyAx - zzAx;
          J[1] = h.mx[1][0] + dzy - xxAy - zzAy;
          J[2] = dzd - xxAz - yyAz;
        } else {
          Cell<float> c;
          Deriv d[3];
#pragma unroll
          for (int f = 0; f < 3; ++f) d[f] = deriv(a, Pz, f);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            c.dA[cc][0] = d[cc].dx;
            c.dA[cc][1] = d[cc].dy;
            c.dA[cc][2] = d[cc].dz;
            c.lapA[cc] = d[cc].xx + d[cc].yy + d[cc].zz;
          }
          c.gdA[0] = d[0].xx + h.mx[0][0] + dzx;
          c.gdA[1] = h.mx[1][0] + d[1].yy + dzy;
          c.gdA[2] = dzd + d[2].zz;
          a_terms<float>(c, a.ph, a.wtab[k], a.wptab[k], B, J, sw);
        }
        float* o = a.bj + (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          o[q * n3] = B[q];
          o[(3 + q) * n3] = J[q];
        }
        if (k >= a.ksw) {
          // layers with swamp terms: J as gd - lap, as in a_terms
          const long long nsw = (long long)(L.nz - a.ksw) * n2;
          float* os = a.sw + (long long)(k - a.ksw) * n2 + (long long)j * L.nx + i;
#pragma unroll
          for (int q = 0; q < 3; ++q) os[q * nsw] = sw[q];
        }
      }
      // all reads of plane k - 3 are done: its slot takes plane k + 5
      __syncthreads();
      if (tid == 0 && k + 5 <= plast) ring.load(&tm, raw, SA, PA * 4, (k + 5 - pbase) & (NRAW - 1), x0, y0, k + 5, AX);
    }
  }
  if (bad) ring.drain(tid, a.ss);
}

// ---------------------------------------------------------------------------
// pass R: box fields u_x, u_y, u_z, ln rho, ln T at 0 .. 4
__global__ void __launch_bounds__(TILE, 2) pass_r_kernel(const __grid_constant__ CUtensorMap tm, const Args a) {
  constexpr int RX = 0, RY = 1, RZ = 2, RL = 3, RT = 4;
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;
  float* wy = raw + NRAW * SR;
  float* wx = wy + TY * WYW;
  Ring ring;
  ring.mbar = (uint64_t*)(wx + WXH * TX);
  const Layout& L = a.L;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  if (halted(a.ss)) return;
  ring.init(tid);

  const int sub = a.sub;
  const bool eval = sub < 0;
  const float dt = eval ? 1.f : (float)a.ss->dt;
  const float alpha = eval ? 0.f : (float)rk_alpha(sub);
  const float beta = eval ? 0.f : (float)rk_beta(sub);
  float rr = 0.f, ss_ = 0.f;
  if (a.ph.bcz == 0) {
    rr = (float)(eval ? a.ss->eval_r : a.ss->r[sub]);
    ss_ = (float)(eval ? a.ss->eval_s : a.ss->s[sub]);
  }
  const FItems items = zm::make_items(tid);
  const int cen = (ty + 3) * BX + tx + 4;
  const int nitems = a.ntx * a.nty * a.nch;
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  bool bad = false;
  Hist h = {};

  for (int item = blockIdx.x; item < nitems && !bad; item += gridDim.x) {
    const int ch = item % a.nch, tile = item / a.nch;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int k0 = ch * a.kchunk, k1 = min(L.nz, k0 + a.kchunk);
    const int pbase = k0 - NG, plast = k1 + NG - 1;
    if (tid == 0)
      for (int p = pbase; p <= min(pbase + NRAW - 1, plast); ++p)
        ring.load(&tm, raw, SR, PR * 4, (p - pbase) & (NRAW - 1), x0, y0, p, UX);
    for (int p = pbase; p < k0 + NG && !bad; ++p) {
      const int s = (p - pbase) & (NRAW - 1);
      bad = !ring.wait(s);
      if (!bad) front(a, items, raw + s * SR, RX, RY, RZ, wy, wx, cen, tx, ty, h);
    }
    for (int k = k0; k < k1 && !bad; ++k) {
      const int i = x0 + tx, j = y0 + ty;
      const bool live = i < L.nx && j < L.ny;
      // per-cell inputs fetched before the front so their latency hides
      // behind it: RK accumulator, A, B, J, swamp terms
      const long long cq = live ? L.at(0, k, j, i) : 0;
      const long long bq = live ? (long long)k * n2 + (long long)j * L.nx + i : 0;
      float dfo[NF], av[3], B[3], J[3], sw[3];
#pragma unroll
      for (int f = 0; f < NF; ++f) dfo[f] = (live && sub > 0) ? __ldg(a.df + cq + (long long)f * L.fs) : 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        av[q] = live ? __ldg(a.fin + cq + (long long)(AX + q) * L.fs) : 0.f;
        B[q] = live ? __ldg(a.bj + bq + q * n3) : 0.f;
        J[q] = live ? __ldg(a.bj + bq + (3 + q) * n3) : 0.f;
        sw[q] = (live && k >= a.ksw)
                    ? __ldg(a.sw + (long long)(k - a.ksw) * n2 + (long long)j * L.nx + i +
                            (long long)q * (L.nz - a.ksw) * n2)
                    : 0.f;
      }
      {
        const int s = (k + NG - pbase) & (NRAW - 1);
        bad = !ring.wait(s);
        if (bad) break;
        front(a, items, raw + s * SR, RX, RY, RZ, wy, wx, cen, tx, ty, h);
      }
      if (live) {
        const int kr = k - pbase;
        const float* Pz[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) Pz[m] = raw + ((kr - 3 + m) & (NRAW - 1)) * SR + cen;
        Deriv d[NFR];
#pragma unroll
        for (int f = 0; f < NFR; ++f) d[f] = deriv(a, Pz, f);
        Cell<float> c;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          c.A[cc] = av[cc];
          c.U[cc] = d[cc].v;
          c.dU[cc][0] = d[cc].dx;
          c.dU[cc][1] = d[cc].dy;
          c.dU[cc][2] = d[cc].dz;
          c.lapU[cc] = d[cc].xx + d[cc].yy + d[cc].zz;
        }
        c.gdU[0] = d[RX].xx + h.mx[0][0] + h.dz(0, a.c1z, a.c2z, a.c3z);
        c.gdU[1] = h.mx[1][0] + d[RY].yy + h.dz(1, a.c1z, a.c2z, a.c3z);
        c.gdU[2] = h.dz(2, a.c1z, a.c2z, a.c3z) + d[RZ].zz;
        c.L = a.bg.lbar[k + NG] + d[RL].v;
        c.Th = a.bg.tbar[k + NG] + d[RT].v;
        c.gL[0] = d[RL].dx;
        c.gL[1] = d[RL].dy;
        c.gL[2] = d[RL].dz + a.bg.dl[k];
        c.gT[0] = d[RT].dx;
        c.gT[1] = d[RT].dy;
        c.gT[2] = d[RT].dz + a.bg.dt[k];
        c.lapL = d[RL].xx + d[RL].yy + d[RL].zz + a.bg.d2l[k];
        c.lapT = d[RT].xx + d[RT].yy + d[RT].zz + a.bg.d2t[k];
        float out[NF];
        rhs_point_bj<float>(c, a.ph, a.wtab[k], B, J, sw, out);
        if (k < a.ph.nc_k1) out[LT] += nc_term<float>(a.ph, a.bg, L.nz, k, c.L, c.Th, nullptr, nullptr);

        float tgx = 0.f, tgy = 0.f;
        const Phys<float>& ph = a.ph;
        if (ph.bcz == 0 && k == 0) {
          const long long q2 = (long long)j * L.nx + i;
          const float vx = a.v0[q2] + ss_ * (a.v1[q2] - a.v0[q2]);
          const float vy = a.v0[n2 + q2] + ss_ * (a.v1[n2 + q2] - a.v0[n2 + q2]);
          tgx = rr * vx;
          tgy = rr * vy;
          out[AX] -= ph.tau_A * (c.A[0] - a.axt[q2]);
          out[AY] -= ph.tau_A * (c.A[1] - a.ayt[q2]);
          out[UX] -= ph.tau_u * (c.U[0] - tgx);
          out[UY] -= ph.tau_u * (c.U[1] - tgy);
          out[UZ] = 0.f;
          out[LR] = 0.f;
        }
        if (ph.bcz == 0 && k == L.nz - 1) out[UZ] = 0.f;
        {
          // periodic images of the cell: offsets computed once for all fields
          const int ox = i < NG ? L.nx : (i >= L.nx - NG ? -L.nx : 0);
          const long long oy = j < NG ? (long long)L.ny * L.mx : (j >= L.ny - NG ? -(long long)L.ny * L.mx : 0);
          const bool small = L.nx < 2 * NG || L.ny < 2 * NG;
          const float vv[NF] = {av[0], av[1], av[2], d[RX].v, d[RY].v, d[RZ].v, d[RL].v, d[RT].v};
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const long long q = cq + (long long)f * L.fs;
            const float dfn = alpha * dfo[f] + dt * out[f];
            if (sub < 2) a.df[q] = dfn;
            if (!eval) {
              const float vn = vv[f] + beta * dfn;
              if (small) {
                zm::store_img(L, a.fout, f, k, j, i, vn);
              } else {
                float* o = a.fout + q;
                o[0] = vn;
                if (ox) o[ox] = vn;
                if (oy) o[oy] = vn;
                if (ox && oy) o[ox + oy] = vn;
              }
            }
          }
        }
        if (ph.bcz == 0 && k == 0) {
          // stateful u_x, u_y ghost rows below the photosphere: nudging only
          for (int m = 1; m <= NG; ++m) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const long long q = L.at(UX + cc, -m, j, i);
              const float u = Pz[3 - m][(RX + cc) * BY * BX];
              const float rh = -ph.tau_u * (u - (cc == 0 ? tgx : tgy));
              const float dfn = (sub > 0 ? alpha * a.df[q] : 0.f) + dt * rh;
              if (sub < 2) a.df[q] = dfn;
              if (!eval) zm::store_img(L, a.fout, UX + cc, -m, j, i, u + beta * dfn);
            }
          }
        }
      }
      // all reads of plane k - 3 are done: its slot takes plane k + 5
      __syncthreads();
      if (tid == 0 && k + 5 <= plast) ring.load(&tm, raw, SR, PR * 4, (k + 5 - pbase) & (NRAW - 1), x0, y0, k + 5, UX);
    }
  }
  if (bad) ring.drain(tid, a.ss);
}

}  // namespace split

size_t rk_split_smem_a() { return split::SMEM_A; }
size_t rk_split_smem_r() { return split::SMEM_R; }

void launch_rk_split(const CUtensorMap* tm_a, const CUtensorMap* tm_r, const Layout& L, const Phys<float>& ph,
                     const Background<float>& bg, const float* fin, float* fout, float* df, float* bj, float* sw,
                     int ksw, const float* wtab, const float* wptab, const Driver& drv, StepState* ss, int sub,
                     double dx, double dy, double dz, cudaStream_t st) {
  // persistent CTAs of pass A and pass R on the current device (their
  // shared-memory limits set there first)
  struct Ctas { int a, r; };
  static PerDevice<Ctas> per_dev;
  const Ctas pc = per_dev.get([] {
    cudaFuncSetAttribute(split::pass_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split::SMEM_A);
    cudaFuncSetAttribute(split::pass_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split::SMEM_R);
    int na = 0, nr = 0;
    const int sms = sm_count();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, split::pass_a_kernel, zm::TILE, split::SMEM_A);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, split::pass_r_kernel, zm::TILE, split::SMEM_R);
    return Ctas{sms * (na > 0 ? na : 1), sms * (nr > 0 ? nr : 1)};
  });
  const int split_ctas[2] = {pc.a, pc.r};

  split::Args a{};
  a.L = L;
  a.ph = ph;
  a.bg = bg;
  a.fin = fin;
  a.fout = fout;
  a.df = df;
  a.bj = bj;
  a.sw = sw;
  a.ksw = ksw;
  a.wtab = wtab;
  a.wptab = wptab;
  a.axt = (const float*)drv.axt;
  a.ayt = (const float*)drv.ayt;
  a.v0 = (const float*)drv.v0;
  a.v1 = (const float*)drv.v1;
  a.ss = ss;
  a.sub = sub;
  a.ntx = (L.nx + zm::TX - 1) / zm::TX;
  a.nty = (L.ny + zm::TY - 1) / zm::TY;
  const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
  const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0, 2.0 / 180.0};
  a.c1x = (float)(W1[1] / dx); a.c2x = (float)(W1[2] / dx); a.c3x = (float)(W1[3] / dx);
  a.c1y = (float)(W1[1] / dy); a.c2y = (float)(W1[2] / dy); a.c3y = (float)(W1[3] / dy);
  a.c1z = (float)(W1[1] / dz); a.c2z = (float)(W1[2] / dz); a.c3z = (float)(W1[3] / dz);
  a.e0x = (float)(W2[0] / (dx * dx)); a.e1x = (float)(W2[1] / (dx * dx));
  a.e2x = (float)(W2[2] / (dx * dx)); a.e3x = (float)(W2[3] / (dx * dx));
  a.e0y = (float)(W2[0] / (dy * dy)); a.e1y = (float)(W2[1] / (dy * dy));
  a.e2y = (float)(W2[2] / (dy * dy)); a.e3y = (float)(W2[3] / (dy * dy));
  a.e0z = (float)(W2[0] / (dz * dz)); a.e1z = (float)(W2[1] / (dz * dz));
  a.e2z = (float)(W2[2] / (dz * dz)); a.e3z = (float)(W2[3] / (dz * dz));
  const int tiles = a.ntx * a.nty;
  const dim3 blk(zm::TX, zm::TY);
  for (int pass = 0; pass < 2; ++pass) {
    const int ctas = split_ctas[pass];
    a.kchunk = zm::zchunk(L.nz, tiles, ctas);
    a.nch = (L.nz + a.kchunk - 1) / a.kchunk;
    const int nitems = tiles * a.nch;
    const int grid = nitems < ctas ? nitems : ctas;
    if (pass == 0)
      split::pass_a_kernel<<<grid, blk, split::SMEM_A, st>>>(*tm_a, a);
    else
      split::pass_r_kernel<<<grid, blk, split::SMEM_R, st>>>(*tm_r, a);
  }
}

}  // namespace mhd
