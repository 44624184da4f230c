// mhd_reduce.cu -- FP64 reductions: the CFL time step and the global
// diagnostics.  Per-cell values are formed in the state precision; block
// partials and the grid-wide result are FP64.  Maxima are order independent
// (the CFL blocks combine theirs by atomicMax); sums are taken in a fixed
// order (per thread, warp tree, block, then one block over the partials) so
// repeated runs give identical bits.
#include <float.h>
#include "mhd_internal.h"

namespace mhd {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// diagnostics grid over (x tiles of 64 cells, y tiles, z chunks); each
// thread walks its z chunk
static inline dim3 red_grid(const Layout& L, int* kchunk) {
  int tx = (L.nx + 63) / 64, ty = (L.ny + 7) / 8;
  int zc = 2432 / (tx * ty);  // about 16 blocks per SM
  if (zc < 1) zc = 1;
  if (zc > L.nz) zc = L.nz;
  if (tx * ty * zc > RED_BLOCKS_MAX) zc = RED_BLOCKS_MAX / (tx * ty) > 0 ? RED_BLOCKS_MAX / (tx * ty) : 1;
  *kchunk = (L.nz + zc - 1) / zc;
  zc = (L.nz + *kchunk - 1) / *kchunk;
  return dim3(tx, ty, zc);
}

// CFL: per cell the advective rate sum|u_i|/dx_i + sqrt(gamma T + B^2/rho)
// sqrt(sum 1/dx_i^2) and the diffusive rate D_max sum 1/dx_i^2, D_max the
// largest of nu, eta + eta_s w, D_rho + chi_rho w, chi_s w + (gamma-1)
// kappa0 T^{5/2}/rho; their maxima over the cells.
//
// Two x-adjacent cells (i even, i + 1) per thread, loaded as 8- or 16-byte
// pairs: the y, z stencils take one pair load per neighbour, the x stencils
// five pair loads for both cells.
template <typename R> struct Pair2;
template <> struct Pair2<float> { using T = float2; };
template <> struct Pair2<double> { using T = double2; };
template <typename R>
__device__ __forceinline__ typename Pair2<R>::T ldp(const R* p) {
  return __ldg(reinterpret_cast<const typename Pair2<R>::T*>(p));
}
// first derivative at p and p + 1 along a stride s that is not x
template <typename R>
__device__ __forceinline__ void d1s_pair(const R* __restrict__ p, int s, R inv, R& r0, R& r1) {
  const auto a1 = ldp(p + s), b1 = ldp(p - s), a2 = ldp(p + 2 * s), b2 = ldp(p - 2 * s);
  const auto a3 = ldp(p + 3 * s), b3 = ldp(p - 3 * s);
  r0 = (W<R>::c1 * (a1.x - b1.x) + W<R>::c2 * (a2.x - b2.x) + W<R>::c3 * (a3.x - b3.x)) * inv;
  r1 = (W<R>::c1 * (a1.y - b1.y) + W<R>::c2 * (a2.y - b2.y) + W<R>::c3 * (a3.y - b3.y)) * inv;
}
// first x derivative at p and p + 1 from the pairs at p - 4 .. p + 4
template <typename R>
__device__ __forceinline__ void d1x_pair(const R* __restrict__ p, R inv, R& r0, R& r1) {
  const auto m4 = ldp(p - 4), m2 = ldp(p - 2), z0 = ldp(p), p2 = ldp(p + 2), p4 = ldp(p + 4);
  r0 = (W<R>::c1 * (z0.y - m2.y) + W<R>::c2 * (p2.x - m2.x) + W<R>::c3 * (p2.y - m4.y)) * inv;
  r1 = (W<R>::c1 * (p2.x - z0.x) + W<R>::c2 * (p2.y - m2.y) + W<R>::c3 * (p4.x - m2.x)) * inv;
}

// Planes k0 .. k0 + nlo - 1, then (blockIdx.z >= nlo) shifted by kgap, so one
// launch can cover the three layers at each end.  Block maxima go by
// atomicMax on the bit patterns (non-negative IEEE doubles order like their
// bits read as unsigned integers, so the result does not depend on the order
// of the blocks) into one of CFL_SLOTS slot pairs, zeroed beforehand.
template <typename R>
__global__ void __launch_bounds__(256) cfl_partial_kernel(Layout L, Phys<R> ph, Background<R> bg,
                                                          const R* __restrict__ f, const R* __restrict__ wtab,
                                                          double* partial, StepState* ss, R sqinv2, int k0, int nlo,
                                                          int kgap) {
  __shared__ R sa[8], sd[8];
  const int i = 2 * (blockIdx.x * 32 + threadIdx.x), j = blockIdx.y * 8 + threadIdx.y;
  const int k = k0 + (int)blockIdx.z + ((int)blockIdx.z >= nlo ? kgap : 0);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (halted(ss)) return;
  // maxima in the state precision (conversion to FP64 is exact and monotonic,
  // so converting the maximum equals the maximum of conversions)
  R mar = R(0), mdr = R(0);
  if (i < L.nx && j < L.ny) {
    const int sy = L.mx;
    const int sz = (int)L.sz();
    // a non-uniform vertical grid: the layer's own inverse spacing dxi/dz in
    // the z derivatives and the advective rate, its own sum of inverse
    // squared spacings in both rates (the finalize then takes 1)
    const bool zg = bg.zm1 != nullptr;
    const R idzk = zg ? bg.zm1[k] : ph.idz;
    const R sqk = zg ? rsqrt_<R>(ph.idx2 + ph.idy2 + idzk * idzk) : sqinv2;
    const R dsc = zg ? ph.idx2 + ph.idy2 + idzk * idzk : R(1);
    const R* pax = f + L.at(AX, k, j, i);
    const R* pay = f + L.at(AY, k, j, i);
    const R* paz = f + L.at(AZ, k, j, i);
    // B = curl A + B_ext (Eq. 6) at both cells
    R dyaz[2], dzay[2], dzax[2], dxaz[2], dxay[2], dyax[2];
    d1s_pair(paz, sy, ph.idy, dyaz[0], dyaz[1]);
    d1s_pair(pay, sz, idzk, dzay[0], dzay[1]);
    d1s_pair(pax, sz, idzk, dzax[0], dzax[1]);
    d1x_pair(paz, ph.idx, dxaz[0], dxaz[1]);
    d1x_pair(pay, ph.idx, dxay[0], dxay[1]);
    d1s_pair(pax, sy, ph.idy, dyax[0], dyax[1]);
    const auto u0 = ldp(f + L.at(UX, k, j, i)), u1 = ldp(f + L.at(UY, k, j, i)), u2 = ldp(f + L.at(UZ, k, j, i));
    const auto plr = ldp(f + L.at(LR, k, j, i)), plt = ldp(f + L.at(LT, k, j, i));
    const R ux[2] = {u0.x, u0.y}, uy[2] = {u1.x, u1.y}, uz[2] = {u2.x, u2.y};
    const R lrs[2] = {plr.x, plr.y}, lts[2] = {plt.x, plt.y};
    const R w = wtab[k];
    const int nc = i + 1 < L.nx ? 2 : 1;
    // A stored about a background: its curl per cell
    R gb[3][2] = {{R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}};
    if (bg.bB) {
      const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz, q3 = (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        gb[cc][0] = bg.bB[cc * n3 + q3];
        if (nc == 2) gb[cc][1] = bg.bB[cc * n3 + q3 + 1];
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c >= nc) break;
      const R B0 = dyaz[c] - dzay[c] + ph.bext[0] + gb[0][c];
      const R B1 = dzax[c] - dxaz[c] + ph.bext[1] + gb[1][c];
      const R B2 = dxay[c] - dyax[c] + ph.bext[2] + gb[2][c];
      const R lr = bg.lbar[k + NG] + lrs[c], lt = bg.tbar[k + NG] + lts[c];
      const R T = rexp<R>(lt), rho1 = rexp<R>(-lr);
      const R B2s = B0 * B0 + B1 * B1 + B2 * B2;
      const R adv = fabs(ux[c]) * ph.idx + fabs(uy[c]) * ph.idy + fabs(uz[c]) * idzk +
                    rsqrt_<R>(ph.gamma * T + B2s * rho1) * sqk;
      R dm = ph.nu;
      dm = fmax(dm, ph.eta + ph.eta_s * w);
      dm = fmax(dm, ph.drho + ph.drho_s * w);
      dm = fmax(dm, ph.chi_s * w + ph.gm1 * ph.kappa0 * rexp<R>(R(2.5) * lt - lr));
      if (zg) dm *= dsc;
      if (!isfinite(adv) || !isfinite(dm)) atomicOr(&ss->nonfinite, 1);
      mar = fmax(mar, adv);
      mdr = fmax(mdr, dm);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mar = fmax(mar, __shfl_xor_sync(0xffffffffu, mar, o));
    mdr = fmax(mdr, __shfl_xor_sync(0xffffffffu, mdr, o));
  }
  if ((tid & 31) == 0) { sa[tid >> 5] = mar; sd[tid >> 5] = mdr; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 8; ++w) { mar = fmax(mar, sa[w]); mdr = fmax(mdr, sd[w]); }
    const int b = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) & (CFL_SLOTS - 1);
    atomicMax((unsigned long long*)&partial[2 * b], (unsigned long long)__double_as_longlong((double)mar));
    atomicMax((unsigned long long*)&partial[2 * b + 1], (unsigned long long)__double_as_longlong((double)mdr));
  }
}

template <typename R>
int launch_cfl_partial(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* f, const R* wtab,
                       double* partial, StepState* ss, CflPlanes planes, bool zero, cudaStream_t st) {
  if (zero) cudaMemsetAsync(partial, 0, sizeof(double) * 2 * CFL_SLOTS, st);
  int k0 = 0, nlo = L.nz, kgap = 0;
  if (planes == CflPlanes::inner) {
    k0 = NG;
    nlo = L.nz - 2 * NG;
  } else if (planes == CflPlanes::ends) {
    nlo = NG;
    kgap = L.nz - 2 * NG;
  }
  const int nk = planes == CflPlanes::ends ? 2 * NG : nlo;
  if (nk > 0) {
    R s2 = (R)sqrt((double)ph.idx2 + (double)ph.idy2 + (double)ph.idz2);
    cfl_partial_kernel<R><<<dim3((L.nx + 63) / 64, (L.ny + 7) / 8, nk), dim3(32, 8), 0, st>>>(
        L, ph, bg, f, wtab, partial, ss, s2, k0, nlo, kgap);
  }
  return CFL_SLOTS;
}

// dt = min(C_adv / max adv, C_diff / max(D_max) / sum 1/dx_i^2) (or dt_fixed);
// then the substep times t + c_s dt with their ramp r and driver weight s
// (Sect. 2.3: linear switch-on, linear interpolation between snapshots).
__global__ void cfl_finalize_kernel(const double* partial, int nblk, StepState* ss, double c_adv,
                                    double c_diff, double dt_fixed, double inv2sum, double t0, double t1,
                                    double t_ramp, int probe) {
  __shared__ double sa[32], sd[32];
  double ma = 0.0, md = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    ma = fmax(ma, partial[2 * b]);
    md = fmax(md, partial[2 * b + 1]);
  }
  ma = warp_max(ma);
  md = warp_max(md);
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = ma; sd[threadIdx.x >> 5] = md; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { ma = fmax(ma, sa[w]); md = fmax(md, sd[w]); }
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else {
    const double d1 = ma > 0.0 ? c_adv / ma : INFINITY;
    const double d2 = md > 0.0 ? c_diff / (md * inv2sum) : INFINITY;
    dt = d1 < d2 ? d1 : d2;
  }
  if (!(dt > 0.0) || !isfinite(dt)) ss->nonfinite = 1;
  if (probe) { ss->probe_dt = dt; return; }
  if (ss->nonfinite) return;
  const double t = ss->t;
  ss->dt = dt;
  for (int s = 0; s < 3; ++s) {
    const double ts = t + rk_c(s) * dt;
    ss->tsub[s] = ts;
    double r = 1.0;
    if (t_ramp > 0.0) r = fmin(fmax(ts / t_ramp, 0.0), 1.0);
    double q = t1 > t0 ? (ts - t0) / (t1 - t0) : 0.0;
    ss->r[s] = r;
    ss->s[s] = fmin(fmax(q, 0.0), 1.0);
  }
  ss->t = t + dt;
  ss->step += 1;
}

void launch_cfl_finalize(const double* partial, int nblk, StepState* ss, double c_adv, double c_diff,
                         double dt_fixed, double inv2sum, double t0, double t1, double t_ramp, int probe,
                         cudaStream_t st) {
  cfl_finalize_kernel<<<1, 256, 0, st>>>(partial, nblk, ss, c_adv, c_diff, dt_fixed, inv2sum, t0, t1,
                                         t_ramp, probe);
}

// Diagnostics, first pass: curl A (Eq. 6, without the uniform B_ext) into the
// scratch fields 0..2 in the state layout.  B_z is formed on the interior
// columns of every plane k = -3 .. nz + 2 (it has no z derivative, and its
// x, y stencils read the periodic rims, which the ghost rules fill on every
// plane); B_x on interior rows and planes for x = -3 .. nx + 2 (it has no x
// derivative), B_y on interior columns and planes for y = -3 .. ny + 2.  So
// the second pass finds every neighbour of its divergence stencil stored,
// the periodic images being computed from the state's images, bit for bit
// equal to the interior values they copy.
template <typename R>
__global__ void __launch_bounds__(256) curl_a_kernel(Layout L, Phys<R> ph, Background<R> bg, const R* __restrict__ f,
                                                     R* __restrict__ bsc) {
  const int i = (int)(blockIdx.x * 32 + threadIdx.x) - NG, j = (int)(blockIdx.y * 8 + threadIdx.y) - NG;
  const int k = (int)blockIdx.z - NG;
  if (i >= L.nx + NG || j >= L.ny + NG) return;
  const bool ix = i >= 0 && i < L.nx, jy = j >= 0 && j < L.ny, kz = k >= 0 && k < L.nz;
  const long long sy = L.sy(), sz = L.sz();
  const R* ax = f + L.at(AX, k, j, i);
  const R* ay = f + L.at(AY, k, j, i);
  const R* az = f + L.at(AZ, k, j, i);
  const long long c = L.at(0, k, j, i);
  const R idzk = (kz && bg.zm1) ? bg.zm1[k] : ph.idz;  // dxi/dz of the layer on a non-uniform grid
  if (ix && jy) bsc[c + 2 * L.fs] = d1(ay, (long long)1, ph.idx) - d1(ax, sy, ph.idy);
  if (jy && kz) bsc[c] = d1(az, sy, ph.idy) - d1(ay, sz, idzk);
  if (ix && kz) bsc[c + L.fs] = d1(ax, sz, idzk) - d1(az, (long long)1, ph.idx);
}

// Second pass: per block 7 values (sums of rho u^2/2, B^2/2, rho T/(gamma-1),
// rho, B_z(k=0), |B_z(k=0)|, and max |div B|) to partial[8 b + q], two
// x-adjacent cells per thread with pair loads.  div B is the centred
// sixth-order divergence of the stored curl A, so it measures how far the
// discrete operators fail to commute; B_ext drops out of it.
template <typename R>
__global__ void __launch_bounds__(256) stats_partial_kernel(Layout L, Phys<R> ph, Background<R> bg,
                                                            const R* __restrict__ f,
                                                            const R* __restrict__ bsc,
                                                            double* partial, int kchunk) {
  __shared__ double sm[8][8];
  const int i = 2 * (blockIdx.x * 32 + threadIdx.x), j = blockIdx.y * 8 + threadIdx.y;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  // a thread's own cells are summed in the state precision with Neumaier
  // compensation (sum + correction carried separately), then taken to FP64:
  // FP64 arithmetic is ~60x slower than FP32 here
  R ps[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, pc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  auto nadd = [&](int q, R x) {
    const R t = ps[q] + x;
    pc[q] += fabs(ps[q]) >= fabs(x) ? (ps[q] - t) + x : (x - t) + ps[q];
    ps[q] = t;
  };
  R dmax = R(0);
  if (i < L.nx && j < L.ny) {
    const int sy = L.mx;
    const int sz = (int)L.sz();
    const int nc = i + 1 < L.nx ? 2 : 1;
    const int k0 = blockIdx.z * kchunk, k1 = min(L.nz, k0 + kchunk);
    for (int k = k0; k < k1; ++k) {
      const R* bx = bsc + L.at(0, k, j, i);
      const R* by = bx + L.fs;
      const R* bz = bx + 2 * L.fs;
      // a non-uniform vertical grid: the layer's dxi/dz and cell extent
      const R idzk = bg.zm1 ? bg.zm1[k] : ph.idz, vk = bg.zcell ? bg.zcell[k] : R(1);
      R dbx[2], dby[2], dbz[2];
      d1x_pair(bx, ph.idx, dbx[0], dbx[1]);
      d1s_pair(by, sy, ph.idy, dby[0], dby[1]);
      d1s_pair(bz, sz, idzk, dbz[0], dbz[1]);
      const auto cx = ldp(bx), cy = ldp(by), cz = ldp(bz);
      const auto u0 = ldp(f + L.at(UX, k, j, i)), u1 = ldp(f + L.at(UY, k, j, i)), u2 = ldp(f + L.at(UZ, k, j, i));
      const auto plr = ldp(f + L.at(LR, k, j, i)), plt = ldp(f + L.at(LT, k, j, i));
      const R bxs[2] = {cx.x, cx.y}, bys[2] = {cy.x, cy.y}, bzs[2] = {cz.x, cz.y};
      const R ux[2] = {u0.x, u0.y}, uy[2] = {u1.x, u1.y}, uz[2] = {u2.x, u2.y};
      const R lrs[2] = {plr.x, plr.y}, lts[2] = {plt.x, plt.y};
      // A stored about a background: its curl per cell (div B stays that of
      // curl A'; div curl A_bg vanishes to FP64 rounding)
      R gb[3][2] = {{R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}};
      if (bg.bB) {
        const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
        const long long q3 = (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          gb[cc][0] = bg.bB[cc * n3 + q3];
          if (nc == 2) gb[cc][1] = bg.bB[cc * n3 + q3 + 1];
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nc) break;
        const R Bx = bxs[c] + ph.bext[0] + gb[0][c], By = bys[c] + ph.bext[1] + gb[1][c],
                Bz = bzs[c] + ph.bext[2] + gb[2][c];
        const R rho = rexp<R>(bg.lbar[k + NG] + lrs[c]);
        const R T = rexp<R>(bg.tbar[k + NG] + lts[c]);
        nadd(0, R(0.5) * rho * (ux[c] * ux[c] + uy[c] * uy[c] + uz[c] * uz[c]) * vk);
        nadd(1, R(0.5) * (Bx * Bx + By * By + Bz * Bz) * vk);
        nadd(2, rho * T * vk);  // / (gamma - 1) once, in the finalize
        nadd(3, rho * vk);
        if (k == 0) {
          nadd(4, Bz);
          nadd(5, fabs(Bz));
        }
        dmax = fmax(dmax, fabs(dbx[c] + dby[c] + dbz[c]));
      }
    }
  }
  for (int q = 0; q < 6; ++q) acc[q] = (double)ps[q] + (double)pc[q];
  acc[6] = (double)dmax;
  for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
  acc[6] = warp_max(acc[6]);
  if ((tid & 31) == 0)
    for (int q = 0; q < 7; ++q) sm[tid >> 5][q] = acc[q];
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 8; ++w) {
      for (int q = 0; q < 6; ++q) acc[q] += sm[w][q];
      acc[6] = fmax(acc[6], sm[w][6]);
    }
    const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    for (int q = 0; q < 7; ++q) partial[8 * b + q] = acc[q];
  }
}

template <typename R>
int launch_stats_partial(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* f, R* bsc,
                         double* partial, cudaStream_t st) {
  dim3 gc((L.nx + 2 * NG + 31) / 32, (L.ny + 2 * NG + 7) / 8, L.nz + 2 * NG);
  curl_a_kernel<R><<<gc, dim3(32, 8), 0, st>>>(L, ph, bg, f, bsc);
  int kchunk;
  dim3 g = red_grid(L, &kchunk);
  stats_partial_kernel<R><<<g, dim3(32, 8), 0, st>>>(L, ph, bg, f, bsc, partial, kchunk);
  return (int)(g.x * g.y * g.z);
}

// fixed-order sums over the block partials; volume sums scaled by dV, the
// photospheric flux sums by dA
__global__ void stats_finalize_kernel(const double* partial, int nblk, StepState* ss, double dv, double da,
                                      double gm1) {
  __shared__ double sm[256][7];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    for (int q = 0; q < 6; ++q) acc[q] += partial[8 * b + q];
    acc[6] = fmax(acc[6], partial[8 * b + 6]);
  }
  for (int q = 0; q < 7; ++q) sm[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      for (int q = 0; q < 6; ++q) sm[threadIdx.x][q] += sm[threadIdx.x + h][q];
      sm[threadIdx.x][6] = fmax(sm[threadIdx.x][6], sm[threadIdx.x + h][6]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sc[7] = {dv, dv, dv / gm1, dv, da, da, 1.0};
    bool bad = false;
    for (int q = 0; q < 7; ++q) {
      ss->stats[q] = sm[0][q] * sc[q];
      if (!isfinite(ss->stats[q])) bad = true;
    }
    ss->stats_t = ss->t;
    if (bad) ss->nonfinite = 1;
  }
}

void launch_stats_finalize(const double* partial, int nblk, StepState* ss, double dv, double da, double gm1,
                           cudaStream_t st) {
  stats_finalize_kernel<<<1, 256, 0, st>>>(partial, nblk, ss, dv, da, gm1);
}

#define INST(R)                                                                                        \
  template int launch_cfl_partial<R>(const Layout&, const Phys<R>&, const Background<R>&, const R*,      \
                                     const R*, double*, StepState*, CflPlanes, bool, cudaStream_t);                     \
  template int launch_stats_partial<R>(const Layout&, const Phys<R>&, const Background<R>&, const R*,    \
                                       R*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mhd
