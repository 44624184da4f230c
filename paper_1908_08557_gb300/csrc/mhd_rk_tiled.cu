// mhd_rk_tiled.cu -- FP32 fused right-hand side + RK3 update, TMA-fed z-march.
//
// A CTA owns a 32 x 8 tile of an xy plane and marches in z over a chunk of
// layers.  Plane p of all 8 fields, with its 3-cell halo, arrives in shared
// memory through one 4D cp.async.bulk.tensor load (box 40 x 14 x 1 x 8: x from
// x0 - 4 so the box starts 16-byte aligned) into an 8-slot ring guarded by
// mbarriers.  Work per plane step (centre k):
//  front (plane k + 3): the quantities whose z derivative gives the xz and
//    yz mixed terms -- D1x A_z, D1y A_z, D1x A_x + D1y A_y and the u
//    analogues -- into a 7-plane ring; the xy mixed terms D1x(D1y A_y),
//    D1y(D1x A_x) (and u) by two passes through shared memory into a 4-plane
//    ring;
//  centre (plane k): first and second derivatives of the 8 fields in x, y, z
//    from the raw ring, D1z of the derived ring, the pointwise physics
//    (rhs_point), boundary rows, the low-storage RK update, and the stores
//    (with periodic images).
// Waits on the ring barriers are bounded; on time-out the CTA sets the
// handle's error word, drains its outstanding copies (bounded) and returns.
#include <cuda.h>

#include "mhd_adjoint_point.cuh"
#include "mhd_internal.h"
#include "mhd_zmarch.cuh"

namespace mhd {
namespace tiled {

using zm::TX;
using zm::TY;
using zm::BX;
using zm::BY;
using zm::WYW;
using zm::WXH;
using zm::TILE;
using zm::FItems;
using zm::make_items;
using zm::mbar_init;
using zm::mbar_wait;
using zm::D1;
using zm::D2;
using zm::store_img;
constexpr int PLANE = NF * BY * BX;          // floats per raw plane
constexpr int NRAW = 8;                      // raw ring: planes k-3 .. k+4
constexpr int NDZ = 6;                       // z-mixed sources per plane
constexpr int NDR = 7;                       // their ring: planes k-3 .. k+3
constexpr int NMX = 4;                       // xy-mixed terms per plane
constexpr int NMR = 4;                       // their ring: planes k .. k+3
constexpr unsigned PLANE_BYTES = PLANE * 4;
constexpr size_t SMEM_FLOATS = (size_t)NRAW * PLANE + NDR * NDZ * TILE + NMR * NMX * TILE + 2 * TY * WYW +
                               2 * WXH * TX;
constexpr size_t SMEM_BYTES = SMEM_FLOATS * 4 + NRAW * 8;

struct Args {
  Layout L;
  Phys<float> ph;
  Background<float> bg;
  float* fout;
  float* df;
  const float* wtab;
  const float* wptab;
  const float* axt;
  const float* ayt;
  const float* v0;
  const float* v1;
  StepState* ss;
  int sub;
  int ntx, nty, nch, kchunk;
  // adjoint mode: D (adjoint of the RK accumulator, padded layout) in, the
  // NCOEF coefficient fields ([NCOEF][nz][ny][nx]) and the driver adjoints out
  const float* dbar;
  float* coef;
  double* thbar;
  float c1x, c2x, c3x, c1y, c2y, c3y, c1z, c2z, c3z;   // D1 weights / spacing
  float e0x, e1x, e2x, e3x, e0y, e1y, e2y, e3y, e0z, e1z, e2z, e3z;  // D2 weights / spacing^2
};

__device__ __forceinline__ void tma_plane(const CUtensorMap* tm, float* dst, uint64_t* bar, int x, int y, int z) {
  zm::tma_plane(tm, dst, bar, PLANE_BYTES, x - 4 + XOFF, y, z, 0);
}

// front processing of one plane: the z-mixed sources and the xy-mixed terms
// (WU = false: A only -- the adjoint reads no second derivative of u)
template <bool WU>
__device__ __forceinline__ void front_plane(const Args& a, const FItems& it, const float* __restrict__ P,
                                            float* __restrict__ D, float* __restrict__ M, float* __restrict__ wy,
                                            float* __restrict__ wx, int cen, int tx, int ty) {
  // F1: D1y of A_y, u_y on the tile plus x halo; D1x of A_x, u_x on the tile
  // plus y halo
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < it.n) {
      if (it.isy[t]) {
        wy[it.dst[t]] = D1(P + AY * BY * BX + it.src[t], BX, a.c1y, a.c2y, a.c3y);
        if (WU) wy[TY * WYW + it.dst[t]] = D1(P + UY * BY * BX + it.src[t], BX, a.c1y, a.c2y, a.c3y);
      } else {
        wx[it.dst[t]] = D1(P + AX * BY * BX + it.src[t], 1, a.c1x, a.c2x, a.c3x);
        if (WU) wx[WXH * TX + it.dst[t]] = D1(P + UX * BY * BX + it.src[t], 1, a.c1x, a.c2x, a.c3x);
      }
    }
  }
  D[0 * TILE] = D1(P + AZ * BY * BX + cen, 1, a.c1x, a.c2x, a.c3x);
  D[1 * TILE] = D1(P + AZ * BY * BX + cen, BX, a.c1y, a.c2y, a.c3y);
  if (WU) {
    D[3 * TILE] = D1(P + UZ * BY * BX + cen, 1, a.c1x, a.c2x, a.c3x);
    D[4 * TILE] = D1(P + UZ * BY * BX + cen, BX, a.c1y, a.c2y, a.c3y);
  }
  __syncthreads();
  // F2: D1x(D1y A_y), D1y(D1x A_x), D1x(D1y u_y), D1y(D1x u_x);
  // D1x A_x + D1y A_y and D1x u_x + D1y u_y
  const float* wyc = wy + ty * WYW + tx + 3;
  const float* wxc = wx + (ty + 3) * TX + tx;
  M[0 * TILE] = D1(wyc, 1, a.c1x, a.c2x, a.c3x);
  M[1 * TILE] = D1(wxc, TX, a.c1y, a.c2y, a.c3y);
  D[2 * TILE] = wxc[0] + wyc[0];
  if (WU) {
    M[2 * TILE] = D1(wyc + TY * WYW, 1, a.c1x, a.c2x, a.c3x);
    M[3 * TILE] = D1(wxc + WXH * TX, TX, a.c1y, a.c2y, a.c3y);
    D[5 * TILE] = wxc[WXH * TX] + wyc[TY * WYW];
  }
  __syncthreads();
}

// ADJ = false: right-hand side + RK update of substep `sub` (sub < 0: store
// the right-hand side only).  ADJ = true: the pointwise adjoint of substep
// `sub` (the input is the ghost-filled substep state): per interior cell the
// NCOEF coefficients of the transposed right-hand side, nothing else stored.
template <bool ADJ>
__global__ void __launch_bounds__(TILE, 1) rk_tiled_kernel(const __grid_constant__ CUtensorMap tm, const Args a) {
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;
  float* dring = raw + NRAW * PLANE;
  float* mring = dring + NDR * NDZ * TILE;
  float* wy = mring + NMR * NMX * TILE;
  float* wx = wy + 2 * TY * WYW;
  uint64_t* mbar = (uint64_t*)(wx + 2 * WXH * TX);

  const Layout& L = a.L;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  if (halted(a.ss)) return;
  if (tid == 0) {
    for (int s = 0; s < NRAW; ++s) mbar_init(&mbar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const int sub = a.sub;
  const bool eval = !ADJ && sub < 0;
  const float dt = eval ? 1.f : (float)a.ss->dt;
  const float alpha = eval ? 0.f : (float)rk_alpha(sub);
  const float beta = eval ? 0.f : (float)rk_beta(sub);
  float rr = 0.f, ss_ = 0.f;
  if (a.ph.bcz == 0) {
    rr = (float)(eval ? a.ss->eval_r : a.ss->r[sub]);
    ss_ = (float)(eval ? a.ss->eval_s : a.ss->s[sub]);
  }
  const FItems items = make_items(tid);
  const int cenoff = (ty + 3) * BX + tx + 4;
  uint32_t phase = 0;   // bit s: parity of the next completion of raw slot s
  uint32_t pending = 0; // bit s: a copy into slot s is in flight
  const int nitems = a.ntx * a.nty * a.nch;
  bool bad = false;     // a ring wait timed out (uniform across the CTA)

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int ch = item % a.nch, tile = item / a.nch;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int k0 = ch * a.kchunk, k1 = min(L.nz, k0 + a.kchunk);
    const int pbase = k0 - NG;
    const int plast = k1 + NG - 1;  // last plane needed
    if (tid == 0) {
      for (int p = pbase; p <= min(pbase + NRAW - 1, plast); ++p) {
        const int s = (p - pbase) & (NRAW - 1);
        tma_plane(&tm, raw + s * PLANE, &mbar[s], x0, y0, p + NG);
        pending |= 1u << s;
      }
    }

    // wait for plane p, then its front processing
#define FRONT(p_)                                                                                   \
  {                                                                                                 \
    const int p__ = (p_);                                                                           \
    const int s__ = (p__ - pbase) & (NRAW - 1);                                                     \
    const bool to__ = !mbar_wait(&mbar[s__], (phase >> s__) & 1u);                                  \
    bad = __syncthreads_or(to__) != 0;                                                              \
    if (!bad) {                                                                                     \
      phase ^= 1u << s__;                                                                           \
      pending &= ~(1u << s__);                                                                      \
      front_plane<!ADJ>(a, items, raw + s__ * PLANE, dring + ((p__ - pbase) % NDR) * NDZ * TILE + tid, \
                  mring + ((p__ - pbase) & (NMR - 1)) * NMX * TILE + tid, wy, wx, cenoff, tx, ty);  \
    }                                                                                               \
  }

    for (int p = pbase; p < k0 + NG && !bad; ++p) FRONT(p);

    for (int k = k0; k < k1 && !bad; ++k) {
      const int i = x0 + tx, j = y0 + ty;
      const bool live = i < L.nx && j < L.ny;
      // RK accumulator of the centre cell, fetched early so its latency hides
      // behind the front processing
      // (adjoint mode: D of the centre cell)
      float dfo[NF];
      {
        const float* dq = (ADJ ? a.dbar : a.df) + (live ? L.at(0, k, j, i) : 0);
#pragma unroll
        for (int f = 0; f < NF; ++f) dfo[f] = (live && (ADJ || sub > 0)) ? __ldg(dq + (long long)f * L.fs) : 0.f;
      }
      FRONT(k + NG);
      if (bad) break;
      if (live) {
        const int cen = (ty + 3) * BX + tx + 4;
        const float* Pk = raw + ((k - pbase) & (NRAW - 1)) * PLANE + cen;
        const int kr = k - pbase;
        const float* const Pz0 = raw + ((kr - 3) & (NRAW - 1)) * PLANE + cen;
        const float* const Pz1 = raw + ((kr - 2) & (NRAW - 1)) * PLANE + cen;
        const float* const Pz2 = raw + ((kr - 1) & (NRAW - 1)) * PLANE + cen;
        const float* const Pz3 = Pk;
        const float* const Pz4 = raw + ((kr + 1) & (NRAW - 1)) * PLANE + cen;
        const float* const Pz5 = raw + ((kr + 2) & (NRAW - 1)) * PLANE + cen;
        const float* const Pz6 = raw + ((kr + 3) & (NRAW - 1)) * PLANE + cen;
        float dx_[NF], dy_[NF], dz_[NF], xx_[NF], yy_[NF], zz_[NF], v_[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const float* p = Pk + f * BY * BX;
          v_[f] = p[0];
          dx_[f] = D1(p, 1, a.c1x, a.c2x, a.c3x);
          dy_[f] = D1(p, BX, a.c1y, a.c2y, a.c3y);
          xx_[f] = D2(p, 1, a.e0x, a.e1x, a.e2x, a.e3x);
          yy_[f] = D2(p, BX, a.e0y, a.e1y, a.e2y, a.e3y);
          const int o = f * BY * BX;
          dz_[f] = a.c1z * (Pz4[o] - Pz2[o]) + a.c2z * (Pz5[o] - Pz1[o]) + a.c3z * (Pz6[o] - Pz0[o]);
          zz_[f] = a.e0z * Pz3[o] + a.e1z * (Pz4[o] + Pz2[o]) + a.e2z * (Pz5[o] + Pz1[o]) +
                   a.e3z * (Pz6[o] + Pz0[o]);
        }
        // D1z of the z-mixed sources
        float mz[NDZ] = {};
        {
          // ring slots of planes k-3 .. k+3 (kr - 3 >= 0 here)
          const float* const Dm3 = dring + ((kr - 3) % NDR) * NDZ * TILE + tid;
          const float* const Dm2 = dring + ((kr - 2) % NDR) * NDZ * TILE + tid;
          const float* const Dm1 = dring + ((kr - 1) % NDR) * NDZ * TILE + tid;
          const float* const Dp1 = dring + ((kr + 1) % NDR) * NDZ * TILE + tid;
          const float* const Dp2 = dring + ((kr + 2) % NDR) * NDZ * TILE + tid;
          const float* const Dp3 = dring + ((kr + 3) % NDR) * NDZ * TILE + tid;
#pragma unroll
          for (int q = 0; q < (ADJ ? 3 : NDZ); ++q) {
            const int o = q * TILE;
            mz[q] = a.c1z * (Dp1[o] - Dm1[o]) + a.c2z * (Dp2[o] - Dm2[o]) + a.c3z * (Dp3[o] - Dm3[o]);
          }
        }
        const float* Mk = mring + ((k - pbase) & (NMR - 1)) * NMX * TILE + tid;
        Cell<float> c;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          c.A[cc] = v_[AX + cc];
          c.U[cc] = v_[UX + cc];
          c.dA[cc][0] = dx_[AX + cc];
          c.dA[cc][1] = dy_[AX + cc];
          c.dA[cc][2] = dz_[AX + cc];
          c.dU[cc][0] = dx_[UX + cc];
          c.dU[cc][1] = dy_[UX + cc];
          c.dU[cc][2] = dz_[UX + cc];
          c.lapA[cc] = xx_[AX + cc] + yy_[AX + cc] + zz_[AX + cc];
          c.lapU[cc] = xx_[UX + cc] + yy_[UX + cc] + zz_[UX + cc];
        }
        c.gdA[0] = xx_[AX] + Mk[0 * TILE] + mz[0];
        c.gdA[1] = Mk[1 * TILE] + yy_[AY] + mz[1];
        c.gdA[2] = mz[2] + zz_[AZ];
        if (ADJ) {
          // the adjoint reads no second derivative of u (its coefficients are
          // nu times the output adjoint); the front skipped them
          c.gdU[0] = c.gdU[1] = c.gdU[2] = 0.f;
        } else {
          c.gdU[0] = xx_[UX] + Mk[2 * TILE] + mz[3];
          c.gdU[1] = Mk[3 * TILE] + yy_[UY] + mz[4];
          c.gdU[2] = mz[5] + zz_[UZ];
        }
        c.L = a.bg.lbar[k + NG] + v_[LR];
        c.Th = a.bg.tbar[k + NG] + v_[LT];
        c.gL[0] = dx_[LR];
        c.gL[1] = dy_[LR];
        c.gL[2] = dz_[LR] + a.bg.dl[k];
        c.gT[0] = dx_[LT];
        c.gT[1] = dy_[LT];
        c.gT[2] = dz_[LT] + a.bg.dt[k];
        c.lapL = xx_[LR] + yy_[LR] + zz_[LR] + a.bg.d2l[k];
        c.lapT = xx_[LT] + yy_[LT] + zz_[LT] + a.bg.d2t[k];
        if constexpr (ADJ) {
          float wo[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) wo[f] = dt * dfo[f];
          const long long q2 = (long long)j * L.nx + i, n2 = (long long)L.nx * L.ny;
          float cf[NCOEF];
          const long long cu = L.at(UX, 0, j, i);
          adjoint_cell<float>(c, a.ph, a.wtab[k], a.wptab[k], wo, dt, k, L.nz, a.dbar + cu, a.dbar + cu + L.fs,
                              L.sz(), a.thbar, q2, n2, a.ss, sub, cf);
          if (k < a.ph.nc_k1) nc_adjoint<float>(a.ph, a.bg, L.nz, k, c.L, c.Th, wo[LT], cf);
          float* co = a.coef + (long long)k * n2 + q2;
          const long long n3 = n2 * L.nz;
#pragma unroll
          for (int q = 0; q < NCOEF; ++q) co[q * n3] = cf[q];
        } else {
          float out[NF];
          rhs_point<float>(c, a.ph, a.wtab[k], a.wptab[k], out);
          if (k < a.ph.nc_k1) out[LT] += nc_term<float>(a.ph, a.bg, L.nz, k, c.L, c.Th, nullptr, nullptr);

          float tgx = 0.f, tgy = 0.f;
          const Phys<float>& ph = a.ph;
          if (ph.bcz == 0 && k == 0) {
            const long long q2 = (long long)j * L.nx + i, n2 = (long long)L.nx * L.ny;
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
            const long long cq = L.at(0, k, j, i);
            const int ox = i < NG ? L.nx : (i >= L.nx - NG ? -L.nx : 0);
            const long long oy = j < NG ? (long long)L.ny * L.mx : (j >= L.ny - NG ? -(long long)L.ny * L.mx : 0);
            const bool small = L.nx < 2 * NG || L.ny < 2 * NG;
  #pragma unroll
            for (int f = 0; f < NF; ++f) {
              const long long q = cq + (long long)f * L.fs;
              const float dfn = alpha * dfo[f] + dt * out[f];
              if (sub < 2) a.df[q] = dfn;
              if (!eval) {
                const float vn = v_[f] + beta * dfn;
                if (small) {
                  store_img(L, a.fout, f, k, j, i, vn);
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
            for (int m = 1; m <= NG; ++m) {
  #pragma unroll
              for (int cc = 0; cc < 2; ++cc) {
                const long long q = L.at(UX + cc, -m, j, i);
                const float u = (m == 1 ? Pz2 : (m == 2 ? Pz1 : Pz0))[(UX + cc) * BY * BX];
                const float rh = -ph.tau_u * (u - (cc == 0 ? tgx : tgy));
                const float dfn = (sub > 0 ? alpha * a.df[q] : 0.f) + dt * rh;
                if (sub < 2) a.df[q] = dfn;
                if (!eval) store_img(L, a.fout, UX + cc, -m, j, i, u + beta * dfn);
              }
            }
          }
        }
      }
      // all reads of plane k - 3 are done: its slot takes plane k + 5
      __syncthreads();
      if (tid == 0 && k + 5 <= plast) {
        const int s = (k + 5 - pbase) & (NRAW - 1);
        tma_plane(&tm, raw + s * PLANE, &mbar[s], x0, y0, k + 5 + NG);
        pending |= 1u << s;
      }
    }
    if (bad) break;
  }
  // `bad` is uniform across the CTA (decided collectively in front())
  if (!bad) return;
  // a ring wait timed out: record it and drain the copies still in flight
  // (bounded) before the CTA's shared memory is released
  if (tid == 0) {
    atomicOr(&a.ss->nonfinite, 2);
    for (int s = 0; s < NRAW; ++s)
      if (pending & (1u << s)) mbar_wait(&mbar[s], (phase >> s) & 1u);
  }
}

}  // namespace tiled

using tiled::Args;

bool rk_tiled_supported() { return true; }

size_t rk_tiled_smem() { return tiled::SMEM_BYTES; }

// persistent CTAs (one per SM) on the current device, after setting the
// kernels' shared-memory limit there
static int tiled_ctas() {
  static PerDevice<int> ctas;
  return ctas.get([] {
    cudaFuncSetAttribute(tiled::rk_tiled_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tiled::SMEM_BYTES);
    cudaFuncSetAttribute(tiled::rk_tiled_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tiled::SMEM_BYTES);
    return sm_count();
  });
}

static Args tiled_args(const Layout& L, const Phys<float>& ph, const Background<float>& bg, const float* wtab,
                       const float* wptab, StepState* ss, int sub, double dx, double dy, double dz) {
  const int sms = tiled_ctas();
  Args a{};
  a.L = L;
  a.ph = ph;
  a.bg = bg;
  a.wtab = wtab;
  a.wptab = wptab;
  a.ss = ss;
  a.sub = sub;
  a.ntx = (L.nx + tiled::TX - 1) / tiled::TX;
  a.nty = (L.ny + tiled::TY - 1) / tiled::TY;
  const int tiles = a.ntx * a.nty;
  a.kchunk = zm::zchunk(L.nz, tiles, sms);
  a.nch = (L.nz + a.kchunk - 1) / a.kchunk;
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
  return a;
}

static int tiled_grid(const Args& a) {
  const int nitems = a.ntx * a.nty * a.nch;
  const int sms = tiled_ctas();
  return nitems < sms ? nitems : sms;
}

void launch_rk_tiled(const CUtensorMap* tm, const Layout& L, const Phys<float>& ph, const Background<float>& bg,
                     float* fout, float* df, const float* wtab, const float* wptab, const Driver& drv,
                     StepState* ss, int sub, double dx, double dy, double dz, cudaStream_t st) {
  Args a = tiled_args(L, ph, bg, wtab, wptab, ss, sub, dx, dy, dz);
  a.fout = fout;
  a.df = df;
  a.axt = (const float*)drv.axt;
  a.ayt = (const float*)drv.ayt;
  a.v0 = (const float*)drv.v0;
  a.v1 = (const float*)drv.v1;
  tiled::rk_tiled_kernel<false><<<tiled_grid(a), dim3(tiled::TX, tiled::TY), tiled::SMEM_BYTES, st>>>(*tm, a);
}

void launch_adj_point_tiled(const CUtensorMap* tm, const Layout& L, const Phys<float>& ph,
                            const Background<float>& bg, const float* dbar, float* coef, double* thbar,
                            const float* wtab, const float* wptab, StepState* ss, int sub, double dx, double dy,
                            double dz, cudaStream_t st) {
  Args a = tiled_args(L, ph, bg, wtab, wptab, ss, sub, dx, dy, dz);
  a.dbar = dbar;
  a.coef = coef;
  a.thbar = thbar;
  tiled::rk_tiled_kernel<true><<<tiled_grid(a), dim3(tiled::TX, tiled::TY), tiled::SMEM_BYTES, st>>>(*tm, a);
}

// Tensor map of one padded FP32 state set: dims (mx, my, mz, 8 fields),
// box (box_x, box_y, 1, box_fields) = one plane of box_fields consecutive
// fields (default 40 x 14: a 32 x 8 tile with its halo).
int make_state_tensor_map(CUtensorMap* tm, const Layout& L, void* base, int box_fields, int box_x, int box_y) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    enc = (EncodeFn)fn;
  }
  cuuint64_t dims[4] = {(cuuint64_t)L.mx, (cuuint64_t)L.my, (cuuint64_t)L.mz, (cuuint64_t)NF};
  cuuint64_t strides[3] = {(cuuint64_t)L.mx * 4, (cuuint64_t)L.my * L.mx * 4, (cuuint64_t)L.fs * 4};
  cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)box_fields};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace mhd
