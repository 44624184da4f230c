// mhd_zmarch.cuh -- pieces shared by the TMA-fed z-march kernels (the fused
// right-hand side / adjoint kernel and the two split right-hand-side passes):
// tile geometry, the mbarrier-guarded TMA plane loads with bounded waits, the
// sixth-order stencils on shared-memory planes, and the periodic-image store.
#pragma once
#include <cuda.h>

#include "mhd_common.cuh"

namespace mhd {
namespace zm {

constexpr int TX = 32, TY = 8;
constexpr int BX = TX + 8;   // box x: x0 - 4 .. x0 + TX + 3 (16-byte aligned start)
constexpr int BY = TY + 6;   // box y: y0 - 3 .. y0 + TY + 2
constexpr int WYW = TX + 6;  // D1y scratch, x halo
constexpr int WXH = TY + 6;  // D1x scratch, y halo
constexpr int TILE = TX * TY;
constexpr int WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(1) : "memory");
}

// one box (BX x BY x 1 x nfields of the tensor map) at (x, y, z, f0)
__device__ __forceinline__ void tma_plane(const CUtensorMap* tm, float* dst, uint64_t* bar, unsigned bytes, int x,
                                          int y, int z, int f0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(sa(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(f0), "r"(sa(bar))
      : "memory");
}

// bounded wait for the given phase parity; false on time-out (after `limit`
// polls, each of which may suspend the thread for a short hardware interval)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = WAIT_LIMIT) {
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ float D1(const float* p, int s, float c1, float c2, float c3) {
  return c1 * (p[s] - p[-s]) + c2 * (p[2 * s] - p[-2 * s]) + c3 * (p[3 * s] - p[-3 * s]);
}
__device__ __forceinline__ float D2(const float* p, int s, float e0, float e1, float e2, float e3) {
  return e0 * p[0] + e1 * (p[s] + p[-s]) + e2 * (p[2 * s] + p[-2 * s]) + e3 * (p[3 * s] + p[-3 * s]);
}

// store v at (k, j, i) and at its periodic x,y images inside the padded
// plane (no local arrays: at most one image per direction for n >= 6, two
// for the smallest grids)
__device__ __forceinline__ void store_img(const Layout& L, float* __restrict__ f, int fl, int k, int j, int i,
                                          float v) {
  const long long base = L.at(fl, k, 0, 0);
  const int mx = L.mx;
  const int xa = i < NG ? i + L.nx : -100, xb = i >= L.nx - NG ? i - L.nx : -100;
  const int ya = j < NG ? j + L.ny : -100, yb = j >= L.ny - NG ? j - L.ny : -100;
  auto put = [&](int jj, int ii) { f[base + (long long)jj * mx + ii] = v; };
  put(j, i);
  if (xa != -100) put(j, xa);
  if (xb != -100) put(j, xb);
  if (ya != -100) {
    put(ya, i);
    if (xa != -100) put(ya, xa);
    if (xb != -100) put(ya, xb);
  }
  if (yb != -100) {
    put(yb, i);
    if (xa != -100) put(yb, xa);
    if (xb != -100) put(yb, xb);
  }
}

// F1 work items of a thread (at most 3): source offset inside a field's box
// plane, destination inside the D1y (wy, tile plus x halo) or D1x (wx, tile
// plus y halo) scratch, and whether it is a wy item
struct FItems {
  int n;
  int src[3], dst[3];
  bool isy[3];
};

__device__ __forceinline__ FItems make_items(int tid) {
  FItems it;
  it.n = 0;
  for (int q = tid; q < TY * WYW + WXH * TX; q += TILE) {
    if (q < TY * WYW) {
      const int r = q / WYW, cx = q - r * WYW;
      it.src[it.n] = (r + 3) * BX + cx + 1;
      it.dst[it.n] = r * WYW + cx;
      it.isy[it.n] = true;
    } else {
      const int q2 = q - TY * WYW;
      const int r = q2 / TX, cx = q2 - r * TX;
      it.src[it.n] = r * BX + cx + 4;
      it.dst[it.n] = r * TX + cx;
      it.isy[it.n] = false;
    }
    ++it.n;
  }
  return it;
}

// z-chunking of a persistent grid of `ctas` CTAs over tiles: balance whole
// waves against the six extra planes each chunk loads before its first
// centre plane; returns the chunk length
inline int zchunk(int nz, int tiles, int ctas) {
  int best = 1;
  double best_eff = 0.0;
  const int maxch = nz / 16 > 1 ? nz / 16 : 1;
  for (int nch = 1; nch <= maxch; ++nch) {
    const int kc = (nz + nch - 1) / nch;
    const int nc = (nz + kc - 1) / kc;
    const long long items = (long long)tiles * nc;
    const long long waves = (items + ctas - 1) / ctas;
    const double eff = (double)items / (double)(waves * ctas) * (double)kc / (double)(kc + 6);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = nch; }
  }
  return (nz + best - 1) / best;
}

}  // namespace zm
}  // namespace mhd
