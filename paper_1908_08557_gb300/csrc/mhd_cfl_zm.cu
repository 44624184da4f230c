// mhd_cfl_zm.cu -- the CFL reduction of the FP32 state over the inner layers
// (those whose z stencils read no ghost plane, k = 3 .. nz - 4) as a z-march:
// one CTA of 128 threads per 32 x 8 tile and z chunk, two x-adjacent cells
// per thread.  The three fields of A arrive plane by plane through TMA (box
// 40 x 14 with the 4 / 3-cell x / y halo, a 4-slot ring guarded by
// mbarriers with bounded waits) for the x and y derivatives of curl A; the
// z derivatives of A_x and A_y come from a register window of the pair's
// seven planes k - 3 .. k + 3, each read once from global memory; u, ln rho,
// ln T are read once per cell.  Every word of the eight fields is read from
// DRAM about once, against about seven times for A_x, A_y and a stencil's
// worth of L1 traffic in the plane-parallel kernel (mhd_reduce.cu).
//
// The arithmetic per cell is that kernel's, term by term and in the same
// order (the stencil sums, the fast-mode and advective rates, the maximum
// diffusivity), and the block maxima go by the same order-independent
// atomicMax on the bit patterns into the same slots, so both kernels give
// the same time step.
#include "mhd_internal.h"
#include "mhd_zmarch.cuh"

namespace mhd {
namespace cflz {

constexpr int TX = zm::TX, TY = zm::TY, BX = zm::BX, BY = zm::BY;
constexpr int NT = TX / 2 * TY;  // 128 threads, one cell pair each
constexpr int NS = 4;            // ring slots: plane k in use, k + 1 .. k + 3 in flight
constexpr int FP = BY * BX;      // floats per field plane of a box
constexpr int PLANE = 3 * FP;    // A_x, A_y, A_z
constexpr int SLOT = (PLANE + 31) / 32 * 32;  // slot stride: a TMA destination starts on 128 bytes
constexpr size_t SMEM_BYTES = (size_t)NS * SLOT * 4 + NS * 8 + 2 * 8 * 4;

// sixth-order first-derivative weights (the plane-parallel kernel's W<float>)
constexpr float C1 = W<float>::c1, C2 = W<float>::c2, C3 = W<float>::c3;

// six CTAs per SM (80 registers): measured 3 % faster at 1024^2 x 256 than
// five (96 registers); eight spill and run 30 % slower
__global__ void __launch_bounds__(NT, 6) cfl_zm_kernel(const __grid_constant__ CUtensorMap tma, Layout L,
                                                    Phys<float> ph, Background<float> bg,
                                                    const float* __restrict__ f, const float* __restrict__ wtab,
                                                    double* partial, StepState* ss, float sqinv2, int ntx, int nty,
                                                    int kchunk, int kbeg, int kend, int wait_limit) {
  extern __shared__ __align__(128) float smem[];
  float* ring = smem;
  uint64_t* mbar = (uint64_t*)(ring + NS * SLOT);
  float* red = (float*)(mbar + NS);  // 2 x 8 warp maxima (4 warps used)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (halted(ss)) return;
  const int tiles = ntx * nty;
  const int tile = blockIdx.x % tiles, ch = blockIdx.x / tiles;
  const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
  const int k0 = kbeg + ch * kchunk, k1 = min(kend, k0 + kchunk);
  const int i = x0 + 2 * tx, j = y0 + ty;
  const bool live = i < L.nx && j < L.ny;
  const int nc = i + 1 < L.nx ? 2 : 1;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) zm::mbar_init(&mbar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0, pending = 0;  // parities; copies in flight (thread 0)
  auto load = [&](int k, int s) {
    zm::tma_plane(&tma, ring + s * SLOT, &mbar[s], PLANE * 4, x0 - 4 + XOFF, y0, k + NG, 0);
    pending |= 1u << s;
  };
  if (tid == 0)
    for (int k = k0; k < k1 && k < k0 + NS; ++k) load(k, k - k0);

  // register window of A_x, A_y at planes k - 3 .. k + 3 (index m + 3)
  const long long q0 = live ? L.at(0, 0, j, i) : 0;  // field 0, layer 0 of the pair
  const long long sz = L.sz();
  auto ld = [&](int fl, int k) {
    return live ? __ldg(reinterpret_cast<const float2*>(f + q0 + fl * L.fs + k * sz)) : make_float2(0.f, 0.f);
  };
  float2 wx[7], wy[7];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    wx[m] = ld(AX, k0 - 3 + m);
    wy[m] = ld(AY, k0 - 3 + m);
  }
  const bool zg = bg.zm1 != nullptr;
  float mar = 0.f, mdr = 0.f;
  bool bad = false;
  int s = 0;
  for (int k = k0; k < k1; ++k) {
    wx[6] = ld(AX, k + 3);
    wy[6] = ld(AY, k + 3);
    const float2 u0 = ld(UX, k), u1 = ld(UY, k), u2 = ld(UZ, k), plr = ld(LR, k), plt = ld(LT, k);
    float gb[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (bg.bB && live) {
      const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz, q3 = (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        gb[cc][0] = bg.bB[cc * n3 + q3];
        if (nc == 2) gb[cc][1] = bg.bB[cc * n3 + q3 + 1];
      }
    }
    const float w = wtab[k];
    const float idzk = zg ? bg.zm1[k] : ph.idz;
    const float sqk = zg ? rsqrt_<float>(ph.idx2 + ph.idy2 + idzk * idzk) : sqinv2;
    const float dsc = zg ? ph.idx2 + ph.idy2 + idzk * idzk : 1.f;
    const bool to = !zm::mbar_wait(&mbar[s], (phase >> s) & 1u, wait_limit);
    if (__syncthreads_or(to)) {
      bad = true;
      break;
    }
    phase ^= 1u << s;
    if (tid == 0) pending &= ~(1u << s);
    if (live) {
      const float* P = ring + s * SLOT + (ty + 3) * BX + 2 * tx + 4;
      auto sp = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
      // first derivative along y (stride BX) and along x at both cells, as the
      // plane-parallel kernel forms them
      auto d1y = [&](const float* p, float& r0, float& r1) {
        const float2 a1 = sp(p + BX), b1 = sp(p - BX), a2 = sp(p + 2 * BX), b2 = sp(p - 2 * BX);
        const float2 a3 = sp(p + 3 * BX), b3 = sp(p - 3 * BX);
        r0 = (C1 * (a1.x - b1.x) + C2 * (a2.x - b2.x) + C3 * (a3.x - b3.x)) * ph.idy;
        r1 = (C1 * (a1.y - b1.y) + C2 * (a2.y - b2.y) + C3 * (a3.y - b3.y)) * ph.idy;
      };
      auto d1x = [&](const float* p, float& r0, float& r1) {
        const float2 m4 = sp(p - 4), m2 = sp(p - 2), z0 = sp(p), p2 = sp(p + 2), p4 = sp(p + 4);
        r0 = (C1 * (z0.y - m2.y) + C2 * (p2.x - m2.x) + C3 * (p2.y - m4.y)) * ph.idx;
        r1 = (C1 * (p2.x - z0.x) + C2 * (p2.y - m2.y) + C3 * (p4.x - m2.x)) * ph.idx;
      };
      float dyaz[2], dzay[2], dzax[2], dxaz[2], dxay[2], dyax[2];
      d1y(P + 2 * FP, dyaz[0], dyaz[1]);
      dzay[0] = (C1 * (wy[4].x - wy[2].x) + C2 * (wy[5].x - wy[1].x) + C3 * (wy[6].x - wy[0].x)) * idzk;
      dzay[1] = (C1 * (wy[4].y - wy[2].y) + C2 * (wy[5].y - wy[1].y) + C3 * (wy[6].y - wy[0].y)) * idzk;
      dzax[0] = (C1 * (wx[4].x - wx[2].x) + C2 * (wx[5].x - wx[1].x) + C3 * (wx[6].x - wx[0].x)) * idzk;
      dzax[1] = (C1 * (wx[4].y - wx[2].y) + C2 * (wx[5].y - wx[1].y) + C3 * (wx[6].y - wx[0].y)) * idzk;
      d1x(P + 2 * FP, dxaz[0], dxaz[1]);
      d1x(P + FP, dxay[0], dxay[1]);
      d1y(P, dyax[0], dyax[1]);
      const float ux[2] = {u0.x, u0.y}, uy[2] = {u1.x, u1.y}, uz[2] = {u2.x, u2.y};
      const float lrs[2] = {plr.x, plr.y}, lts[2] = {plt.x, plt.y};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nc) break;
        const float B0 = dyaz[c] - dzay[c] + ph.bext[0] + gb[0][c];
        const float B1 = dzax[c] - dxaz[c] + ph.bext[1] + gb[1][c];
        const float B2 = dxay[c] - dyax[c] + ph.bext[2] + gb[2][c];
        const float lr = bg.lbar[k + NG] + lrs[c], lt = bg.tbar[k + NG] + lts[c];
        const float T = rexp<float>(lt), rho1 = rexp<float>(-lr);
        const float B2s = B0 * B0 + B1 * B1 + B2 * B2;
        const float adv = fabsf(ux[c]) * ph.idx + fabsf(uy[c]) * ph.idy + fabsf(uz[c]) * idzk +
                          rsqrt_<float>(ph.gamma * T + B2s * rho1) * sqk;
        float dm = ph.nu;
        dm = fmaxf(dm, ph.eta + ph.eta_s * w);
        dm = fmaxf(dm, ph.drho + ph.drho_s * w);
        dm = fmaxf(dm, ph.chi_s * w + ph.gm1 * ph.kappa0 * rexp<float>(2.5f * lt - lr));
        if (zg) dm *= dsc;
        if (!isfinite(adv) || !isfinite(dm)) atomicOr(&ss->nonfinite, 1);
        mar = fmaxf(mar, adv);
        mdr = fmaxf(mdr, dm);
      }
    }
    // every thread is past plane k: its slot takes plane k + NS
    __syncthreads();
    if (tid == 0 && k + NS < k1) load(k + NS, s);
    s = s + 1 == NS ? 0 : s + 1;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      wx[m] = wx[m + 1];
      wy[m] = wy[m + 1];
    }
  }
  if (bad) {
    // a ring wait timed out: record it and drain the copies in flight (bounded)
    if (tid == 0) {
      atomicOr(&ss->nonfinite, 2);
      for (int q = 0; q < NS; ++q)
        if (pending & (1u << q)) zm::mbar_wait(&mbar[q], (phase >> q) & 1u, wait_limit);
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mar = fmaxf(mar, __shfl_xor_sync(0xffffffffu, mar, o));
    mdr = fmaxf(mdr, __shfl_xor_sync(0xffffffffu, mdr, o));
  }
  if ((tid & 31) == 0) {
    red[tid >> 5] = mar;
    red[8 + (tid >> 5)] = mdr;
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 1; q < NT / 32; ++q) {
      mar = fmaxf(mar, red[q]);
      mdr = fmaxf(mdr, red[8 + q]);
    }
    const int b = blockIdx.x & (CFL_SLOTS - 1);
    atomicMax((unsigned long long*)&partial[2 * b], (unsigned long long)__double_as_longlong((double)mar));
    atomicMax((unsigned long long*)&partial[2 * b + 1], (unsigned long long)__double_as_longlong((double)mdr));
  }
}

}  // namespace cflz

int launch_cfl_inner_zm(const CUtensorMap* tma, const Layout& L, const Phys<float>& ph, const Background<float>& bg,
                        const float* f, const float* wtab, double* partial, StepState* ss, bool zero,
                        cudaStream_t st) {
  if (zero) cudaMemsetAsync(partial, 0, sizeof(double) * 2 * CFL_SLOTS, st);
  const int kbeg = NG, kend = L.nz - NG;
  if (kend <= kbeg) return CFL_SLOTS;
  static PerDevice<int> resident;
  const int res = resident.get([] {
    cudaFuncSetAttribute((const void*)cflz::cfl_zm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cflz::SMEM_BYTES);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cflz::cfl_zm_kernel, cflz::NT, cflz::SMEM_BYTES);
    return (per_sm > 0 ? per_sm : 1) * sm_count();
  });
  const int ntx = (L.nx + cflz::TX - 1) / cflz::TX, nty = (L.ny + cflz::TY - 1) / cflz::TY;
  const long long tiles = (long long)ntx * nty;
  // chunks of 8 .. 64 layers, about four waves of resident CTAs in all
  const int nk = kend - kbeg;
  long long kc = tiles * nk / (4LL * res);
  kc = kc < 8 ? 8 : (kc > 64 ? 64 : kc);
  const int kchunk = (int)kc;
  const int nch = (nk + kchunk - 1) / kchunk;
  const float s2 = (float)sqrt((double)ph.idx2 + (double)ph.idy2 + (double)ph.idz2);
  cflz::cfl_zm_kernel<<<(unsigned)(tiles * nch), cflz::NT, cflz::SMEM_BYTES, st>>>(
      *tma, L, ph, bg, f, wtab, partial, ss, s2, ntx, nty, kchunk, kbeg, kend, zm::WAIT_LIMIT);
  return CFL_SLOTS;
}

}  // namespace mhd
