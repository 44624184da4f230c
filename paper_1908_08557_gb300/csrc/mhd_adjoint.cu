// mhd_adjoint.cu -- hand-written adjoint (transposed linearisation) of one
// low-storage RK3 step with a frozen time step.
//
// Forward substep s:  r_s = R(f_s) = RHS(ghost_fill(f_s)),
//                     df_{s+1} = alpha_s df_s + dt r_s,  f_{s+1} = f_s + beta_s df_{s+1}.
// Reverse, s = 2, 1, 0 (F = adjoint of the state, D = adjoint of df):
//                     D += beta_s F;  W = dt D;  F += (dR/df)^T W;  D = alpha_s D,
// with the driver adjoints accumulated from W at the photosphere.
// (dR/df)^T W is assembled from
//  1. adj_point_kernel: per interior cell, the transpose of the pointwise
//     physics (rhs_point) and of the boundary rows / nudging terms, giving
//     40 coefficients: adjoints of the cell values and of every derivative
//     the right-hand side used (first, second, mixed);
//  2. the gather (adj_gather_kernel, or gd_fold_kernel + the tiled
//     gather_tiled_kernel): the transposed stencils (D1^T = -D1, D2^T = D2,
//     (D1_a D1_b)^T = D1_a D1_b, periodic in x and y) applied to the
//     coefficient fields, at interior points and z ghost layers, plus the
//     nudging value adjoints of A and of the u ghost rows;
//  3. adj_bc_kernel: the transpose of the pointwise ghost rules (Eqs. 8, 11,
//     13, closed u_z, symmetric u_hor), routing ghost adjoints into the
//     interior; the potential-field ghosts are transposed by the FFT kernels
//     (the Eq. 17 multiplier is real and even, so it is its own transpose).
#include "mhd_adjoint_point.cuh"
#include "mhd_internal.h"

namespace mhd {

template <typename R>
struct AdjPointArgs {
  Layout L;
  Phys<R> ph;
  Background<R> bg;
  const R* g;        // ghost-filled forward state of the substep (perturbation storage)
  const R* dbar;     // adjoint of df (padded layout)
  R* coef;           // [NCOEF][nz][ny][nx]
  double* thbar;     // [6][ny][nx]: A_target x, y; v0 x, y; v1 x, y
  const R* wtab;
  const R* wptab;
  const StepState* ss;
  int sub;
};

template <typename R>
__global__ void __launch_bounds__(128) adj_point_kernel(AdjPointArgs<R> a) {
  const Layout& L = a.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  if (halted(a.ss)) return;
  const Phys<R>& ph = a.ph;
  const long long st[3] = {1, L.sy(), L.sz()};
  const R inv[3] = {ph.idx, ph.idy, ph.idz};
  const R inv2[3] = {ph.idx2, ph.idy2, ph.idz2};
  const R* base[NF];
  for (int fl = 0; fl < NF; ++fl) base[fl] = a.g + L.at(fl, k, j, i);
  // the cell record, exactly as the forward kernels build it
  Cell<R> c;
  for (int cc = 0; cc < 3; ++cc) {
    const R* pa = base[AX + cc];
    const R* pu = base[UX + cc];
    c.A[cc] = *pa;
    c.U[cc] = *pu;
    c.lapA[cc] = R(0);
    c.lapU[cc] = R(0);
    for (int ax = 0; ax < 3; ++ax) {
      c.dA[cc][ax] = d1(pa, st[ax], inv[ax]);
      c.dU[cc][ax] = d1(pu, st[ax], inv[ax]);
      c.lapA[cc] += d2(pa, st[ax], inv2[ax]);
      c.lapU[cc] += d2(pu, st[ax], inv2[ax]);
    }
  }
  for (int ax = 0; ax < 3; ++ax) {
    R sa = R(0), su = R(0);
    for (int cc = 0; cc < 3; ++cc) {
      if (cc == ax) {
        sa += d2(base[AX + cc], st[ax], inv2[ax]);
        su += d2(base[UX + cc], st[ax], inv2[ax]);
      } else {
        sa += d11(base[AX + cc], st[ax], st[cc], inv[ax], inv[cc]);
        su += d11(base[UX + cc], st[ax], st[cc], inv[ax], inv[cc]);
      }
    }
    c.gdA[ax] = sa;
    c.gdU[ax] = su;
  }
  c.L = a.bg.lbar[k + NG] + *base[LR];
  c.Th = a.bg.tbar[k + NG] + *base[LT];
  c.lapL = R(0);
  c.lapT = R(0);
  for (int ax = 0; ax < 3; ++ax) {
    c.gL[ax] = d1(base[LR], st[ax], inv[ax]);
    c.gT[ax] = d1(base[LT], st[ax], inv[ax]);
    c.lapL += d2(base[LR], st[ax], inv2[ax]);
    c.lapT += d2(base[LT], st[ax], inv2[ax]);
  }
  c.gL[2] += a.bg.dl[k];
  c.lapL += a.bg.d2l[k];
  c.gT[2] += a.bg.dt[k];
  c.lapT += a.bg.d2t[k];

  const R dt = R(a.ss->dt);
  R wo[NF];
  for (int fl = 0; fl < NF; ++fl) wo[fl] = dt * a.dbar[L.at(fl, k, j, i)];
  const long long q2 = (long long)j * L.nx + i, n2 = (long long)L.nx * L.ny;
  R cf[NCOEF];
  adjoint_cell<R>(c, ph, a.wtab[k], a.wptab[k], wo, dt, k, L.nz, a.dbar + L.at(UX, 0, j, i),
                  a.dbar + L.at(UY, 0, j, i), L.sz(), a.thbar, q2, n2, a.ss, a.sub, cf);
  if (k < ph.nc_k1) nc_adjoint<R>(ph, a.bg, L.nz, k, c.L, c.Th, wo[LT], cf);
  const long long n3 = n2 * L.nz, cq = (long long)k * n2 + q2;
  for (int q = 0; q < NCOEF; ++q) a.coef[q * n3 + cq] = cf[q];
}

// ---------------------------------------------------------------------------
template <typename R>
struct AdjGatherArgs {
  Layout L;
  Phys<R> ph;
  const R* coef;
  const R* dbar;
  R* gbar;           // output: adjoint of the ghost-filled input (padded layout)
  const StepState* ss;
};

template <typename R>
__device__ __forceinline__ R cget(const R* __restrict__ coef, int q, int k, int j, int i, int nx, int ny, int nz) {
  if (k < 0 || k >= nz) return R(0);
  i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
  j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
  return __ldg(coef + (((long long)q * nz + k) * ny + j) * nx + i);
}

// transposed first derivative along axis ax of coefficient q at (k, j, i)
template <typename R>
__device__ __forceinline__ R t_d1(const R* coef, int q, int k, int j, int i, int ax, int nx, int ny, int nz, R inv) {
  R s = R(0);
  const R cw[4] = {R(0), W<R>::c1, W<R>::c2, W<R>::c3};
  for (int m = 1; m <= 3; ++m) {
    const int di = ax == 0 ? m : 0, dj = ax == 1 ? m : 0, dk = ax == 2 ? m : 0;
    s += cw[m] * (cget(coef, q, k - dk, j - dj, i - di, nx, ny, nz) - cget(coef, q, k + dk, j + dj, i + di, nx, ny, nz));
  }
  return s * inv;
}
template <typename R>
__device__ __forceinline__ R t_d2(const R* coef, int q, int k, int j, int i, int ax, int nx, int ny, int nz, R inv2) {
  const R ew[4] = {W<R>::e0, W<R>::e1, W<R>::e2, W<R>::e3};
  R s = ew[0] * cget(coef, q, k, j, i, nx, ny, nz);
  for (int m = 1; m <= 3; ++m) {
    const int di = ax == 0 ? m : 0, dj = ax == 1 ? m : 0, dk = ax == 2 ? m : 0;
    s += ew[m] * (cget(coef, q, k - dk, j - dj, i - di, nx, ny, nz) + cget(coef, q, k + dk, j + dj, i + di, nx, ny, nz));
  }
  return s * inv2;
}
// transposed mixed derivative D1_a D1_b (its own transpose)
template <typename R>
__device__ __forceinline__ R t_d11(const R* coef, int q, int k, int j, int i, int a, int b, int nx, int ny, int nz,
                                   R ia, R ib) {
  const R cw[4] = {R(0), W<R>::c1, W<R>::c2, W<R>::c3};
  R s = R(0);
  for (int m = 1; m <= 3; ++m)
    for (int n = 1; n <= 3; ++n) {
      int d[2][3] = {{0, 0, 0}, {0, 0, 0}};
      d[0][a] = m;
      d[1][b] = n;
      const int pi = d[0][0] + d[1][0], pj = d[0][1] + d[1][1], pk = d[0][2] + d[1][2];
      const int qi = d[0][0] - d[1][0], qj = d[0][1] - d[1][1], qk = d[0][2] - d[1][2];
      const R v = cget(coef, q, k + pk, j + pj, i + pi, nx, ny, nz) - cget(coef, q, k + qk, j + qj, i + qi, nx, ny, nz) -
                  cget(coef, q, k - qk, j - qj, i - qi, nx, ny, nz) + cget(coef, q, k - pk, j - pj, i - pi, nx, ny, nz);
      s += cw[m] * cw[n] * v;
    }
  return s * ia * ib;
}

template <typename R>
__global__ void __launch_bounds__(128) adj_gather_kernel(AdjGatherArgs<R> a) {
  const Layout& L = a.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = (int)blockIdx.z - NG;
  if (i >= L.nx || j >= L.ny) return;
  if (halted(a.ss)) return;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const Phys<R>& ph = a.ph;
  const R inv[3] = {ph.idx, ph.idy, ph.idz};
  const R inv2[3] = {ph.idx2, ph.idy2, ph.idz2};
  const bool inside = k >= 0 && k < nz;
  const R dt = R(a.ss->dt);
  for (int cc = 0; cc < 3; ++cc) {
    for (int grp = 0; grp < 2; ++grp) {  // grp 0: A_c, grp 1: u_c
      // gd(u) coefficients are the lap(u) ones divided by 3
      const int qd = grp == 0 ? CDA : CDU, ql = grp == 0 ? CLA : CLU, qg = grp == 0 ? CGA : CLU;
      const R gs = grp == 0 ? R(1) : R(1.0 / 3.0);
      const int fl = (grp == 0 ? AX : UX) + cc;
      R s = (inside && grp == 1) ? cget(a.coef, CV + fl, k, j, i, nx, ny, nz) : R(0);
      for (int ax = 0; ax < 3; ++ax) {
        s += t_d1(a.coef, qd + 3 * cc + ax, k, j, i, ax, nx, ny, nz, inv[ax]);
        s += t_d2(a.coef, ql + cc, k, j, i, ax, nx, ny, nz, inv2[ax]);
      }
      s += gs * t_d2(a.coef, qg + cc, k, j, i, cc, nx, ny, nz, inv2[cc]);
      for (int ax = 0; ax < 3; ++ax)
        if (ax != cc) s += gs * t_d11(a.coef, qg + ax, k, j, i, ax, cc, nx, ny, nz, inv[ax], inv[cc]);
      // photospheric nudging of A_x, A_y (Eq. 4): value adjoint -tau_A dt D
      if (ph.bcz == 0 && k == 0 && grp == 0 && cc < 2) s -= ph.tau_A * dt * a.dbar[L.at(fl, k, j, i)];
      a.gbar[L.at(fl, k, j, i)] = s;
    }
  }
  for (int grp = 0; grp < 2; ++grp) {  // ln rho, ln T
    const int qg = grp == 0 ? CGL : CGT, ql = grp == 0 ? CLL : CLT, fl = grp == 0 ? LR : LT;
    R s = inside ? cget(a.coef, CV + fl, k, j, i, nx, ny, nz) : R(0);
    for (int ax = 0; ax < 3; ++ax) {
      s += t_d1(a.coef, qg + ax, k, j, i, ax, nx, ny, nz, inv[ax]);
      s += t_d2(a.coef, ql, k, j, i, ax, nx, ny, nz, inv2[ax]);
    }
    a.gbar[L.at(fl, k, j, i)] = s;
  }
  // stateful horizontal-velocity ghost rows: their own nudging term
  if (ph.bcz == 0 && k < 0) {
    for (int cc = 0; cc < 2; ++cc) {
      const long long q = L.at(UX + cc, k, j, i);
      a.gbar[q] -= ph.tau_u * dt * a.dbar[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Transpose of the pointwise ghost rules (per column, interior x,y): ghost
// adjoints are routed into the layers they were computed from.
template <typename R>
__global__ void adj_bc_kernel(Layout L, Phys<R> ph, Background<R> bg, const R* __restrict__ g, R* __restrict__ gbar,
                              R dz, const StepState* ss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L.nx * L.ny) return;
  if (halted(ss)) return;
  const int i = q % L.nx, j = q / L.nx;
  const int kt = L.nz - 1;
  const R dzg = dz * ph.gz;
  // bottom: ln T recursion (ln rho ghosts are constants)
  {
    const R th0 = bg.tbar[NG] + g[L.at(LT, 0, j, i)];
    const R thm1 = bg.tbar[NG - 1] + g[L.at(LT, -1, j, i)];
    const R thm2 = bg.tbar[NG - 2] + g[L.at(LT, -2, j, i)];
    const R a3 = gbar[L.at(LT, -3, j, i)];
    const R a2 = gbar[L.at(LT, -2, j, i)] + a3 * (R(1) + dzg * rexp<R>(-thm2));
    const R a1 = gbar[L.at(LT, -1, j, i)] + a2 * (R(1) + dzg * rexp<R>(-thm1));
    gbar[L.at(LT, 0, j, i)] += a1 * (R(1) + dzg * rexp<R>(-th0));
    gbar[L.at(LR, 0, j, i)] += a1;
    for (int m = 1; m <= NG; ++m) gbar[L.at(UZ, m, j, i)] -= gbar[L.at(UZ, -m, j, i)];
  }
  // top
  {
    const R Ttop = rexp<R>(bg.tbar[NG + kt] + g[L.at(LT, kt, j, i)]);
    R bth = R(0);
    for (int m = 1; m <= NG; ++m) {
      gbar[L.at(LT, kt - m, j, i)] += gbar[L.at(LT, kt + m, j, i)];
      const R bl = gbar[L.at(LR, kt + m, j, i)];
      gbar[L.at(LR, kt - m, j, i)] += bl;
      bth -= bl * (R(2 * m) * dz) * ph.gz / Ttop;
      gbar[L.at(UZ, kt - m, j, i)] -= gbar[L.at(UZ, kt + m, j, i)];
      gbar[L.at(UX, kt - m, j, i)] += gbar[L.at(UX, kt + m, j, i)];
      gbar[L.at(UY, kt - m, j, i)] += gbar[L.at(UY, kt + m, j, i)];
    }
    gbar[L.at(LT, kt, j, i)] += bth;
  }
}

// Elementwise adjoint updates over the cells that carry state (interior, and
// the u_x, u_y ghost layers below the photosphere), 16 bytes per thread and
// row-contiguous (nx is a multiple of 4):
//   mode 0, start of a sweep: D = beta_2 F
//   mode 1, end of substep s: F += G;  D = alpha_s D + beta F, with beta = beta_{s-1},
//           and for s = 0 (alpha_0 = 0) beta = beta_2: the next step's first update
// Interior layers klo <= k < khi are skipped (the tiled gather updates them).
template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
};
template <typename V, typename R>
__device__ __forceinline__ R& vat(V& v, int e) {
  return reinterpret_cast<R*>(&v)[e];
}

template <typename R>
__global__ void __launch_bounds__(256) adj_update_kernel(Layout L, R* __restrict__ fbar, R* __restrict__ dbar,
                                                         const R* __restrict__ gbar, R alpha, R beta, int mode,
                                                         int klo, int khi, const StepState* ss) {
  using V = typename Vec16<R>::T;
  constexpr int E = Vec16<R>::N;
  if (halted(ss)) return;
  const unsigned ny = L.ny, vpr = L.nx / E, nyz = (unsigned)(L.nz - (khi - klo)) * ny, ngy = NG * ny;
  const unsigned nrow_int = NF * nyz;
  const unsigned nvec = (nrow_int + 2 * ngy) * vpr;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nvec; q += gridDim.x * blockDim.x) {
    const unsigned row = q / vpr, v = q - row * vpr;
    int f, k, j;
    if (row < nrow_int) {
      f = row / nyz;
      const unsigned r = row - f * nyz;
      k = r / ny;
      j = r - k * ny;
      if (k >= klo) k += khi - klo;
    } else {
      unsigned r = row - nrow_int;
      const unsigned g = r / ngy;
      f = UX + (int)g;
      r -= g * ngy;
      k = -1 - (int)(r / ny);
      j = r % ny;
    }
    const long long p = L.at(f, k, j, (int)(v * E));
    V fv = *reinterpret_cast<const V*>(fbar + p);
    V dv;
    if (mode == 0) {
#pragma unroll
      for (int e = 0; e < E; ++e) vat<V, R>(dv, e) = beta * vat<V, R>(fv, e);
    } else {
      const V gv = *reinterpret_cast<const V*>(gbar + p);
      dv = *reinterpret_cast<const V*>(dbar + p);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        vat<V, R>(fv, e) += vat<V, R>(const_cast<V&>(gv), e);
        vat<V, R>(dv, e) = alpha * vat<V, R>(dv, e) + beta * vat<V, R>(fv, e);
      }
      *reinterpret_cast<V*>(fbar + p) = fv;
    }
    *reinterpret_cast<V*>(dbar + p) = dv;
  }
}

// ---------------------------------------------------------------------------
// B_z = D1x A_y - D1y A_x on layer k of an interior-packed state (periodic),
// and its transpose: lam_Ay = -D1x(bbar), lam_Ax = +D1y(bbar).
template <typename R>
__global__ void bz_plane_kernel(int nx, int ny, int nz, int k, R idx, R idy, const R* __restrict__ st,
                                R* __restrict__ out, int adjoint, const R* __restrict__ bbar, R* __restrict__ lam) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nx * ny) return;
  const int i = q % nx, j = q / nx;
  const long long n2 = (long long)nx * ny, n3 = n2 * nz;
  const R cw[4] = {R(0), W<R>::c1, W<R>::c2, W<R>::c3};
  auto at = [&](const R* p, int jj, int ii) -> R {
    ii = (ii % nx + nx) % nx;
    jj = (jj % ny + ny) % ny;
    return p[(long long)jj * nx + ii];
  };
  if (!adjoint) {
    const R* ax = st + 0 * n3 + (long long)k * n2;
    const R* ay = st + 1 * n3 + (long long)k * n2;
    R dx = R(0), dy = R(0);
    for (int m = 1; m <= 3; ++m) {
      dx += cw[m] * (at(ay, j, i + m) - at(ay, j, i - m));
      dy += cw[m] * (at(ax, j + m, i) - at(ax, j - m, i));
    }
    out[q] = dx * idx - dy * idy;
  } else {
    R gx = R(0), gy = R(0);
    for (int m = 1; m <= 3; ++m) {
      gx += cw[m] * (at(bbar, j, i - m) - at(bbar, j, i + m));  // D1x^T
      gy += cw[m] * (at(bbar, j - m, i) - at(bbar, j + m, i));  // D1y^T
    }
    lam[1 * n3 + (long long)k * n2 + q] = gx * idx;
    lam[0 * n3 + (long long)k * n2 + q] = -gy * idy;
  }
}

// adjoint state <-> interior layout (no background: these are adjoints);
// on the way out the stateful u_x, u_y ghost adjoints are folded onto the
// photospheric layer (the ghosts are initialised from it)
template <typename R>
__global__ void adj_pack_kernel(Layout L, int bcz, const R* __restrict__ fbar, R* __restrict__ out) {
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3 * NF;
       q += (long long)gridDim.x * blockDim.x) {
    const int fl = (int)(q / n3);
    const long long r = q - (long long)fl * n3;
    const int k = (int)(r / n2);
    const long long rem = r - (long long)k * n2;
    const int j = (int)(rem / L.nx), i = (int)(rem - (long long)j * L.nx);
    R v = fbar[L.at(fl, k, j, i)];
    if (bcz == 0 && k == 0 && (fl == UX || fl == UY))
      for (int m = 1; m <= NG; ++m) v += fbar[L.at(fl, -m, j, i)];
    out[q] = v;
  }
}

template <typename R>
__global__ void adj_unpack_kernel(Layout L, const R* __restrict__ in, R* __restrict__ fbar) {
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3 * NF;
       q += (long long)gridDim.x * blockDim.x) {
    const int fl = (int)(q / n3);
    const long long r = q - (long long)fl * n3;
    const int k = (int)(r / n2);
    const long long rem = r - (long long)k * n2;
    const int j = (int)(rem / L.nx), i = (int)(rem - (long long)j * L.nx);
    fbar[L.at(fl, k, j, i)] = in[q];
  }
}

template <typename R>
__global__ void d2r_kernel(const double* __restrict__ in, R* __restrict__ out, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (R)in[q];
}

template <typename R>
void launch_adj_pack(const Layout& L, int bcz, const R* fbar, R* out, cudaStream_t st) {
  adj_pack_kernel<R><<<1216, 256, 0, st>>>(L, bcz, fbar, out);
}
template <typename R>
void launch_adj_unpack(const Layout& L, const R* in, R* fbar, cudaStream_t st) {
  adj_unpack_kernel<R><<<1216, 256, 0, st>>>(L, in, fbar);
}
template <typename R>
void launch_d2r(const double* in, R* out, long long n, cudaStream_t st) {
  d2r_kernel<R><<<304, 256, 0, st>>>(in, out, n);
}

// ---------------------------------------------------------------------------
template <typename R>
void launch_adj_point(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* g, const R* dbar, R* coef,
                      double* thbar, const R* wtab, const R* wptab, const StepState* ss, int sub, cudaStream_t st) {
  AdjPointArgs<R> a;
  a.L = L; a.ph = ph; a.bg = bg; a.g = g; a.dbar = dbar; a.coef = coef; a.thbar = thbar;
  a.wtab = wtab; a.wptab = wptab; a.ss = ss; a.sub = sub;
  dim3 blk(32, 4, 1), grd((L.nx + 31) / 32, (L.ny + 3) / 4, L.nz);
  adj_point_kernel<R><<<grd, blk, 0, st>>>(a);
}

template <typename R>
void launch_adj_gather(const Layout& L, const Phys<R>& ph, const R* coef, const R* dbar, R* gbar, const StepState* ss,
                       cudaStream_t st) {
  AdjGatherArgs<R> a;
  a.L = L; a.ph = ph; a.coef = coef; a.dbar = dbar; a.gbar = gbar; a.ss = ss;
  dim3 blk(32, 4, 1), grd((L.nx + 31) / 32, (L.ny + 3) / 4, L.nz + 2 * NG);
  adj_gather_kernel<R><<<grd, blk, 0, st>>>(a);
}

template <typename R>
void launch_adj_bc(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* g, R* gbar, R dz,
                   const StepState* ss, cudaStream_t st) {
  const int n = L.nx * L.ny;
  adj_bc_kernel<R><<<(n + 127) / 128, 128, 0, st>>>(L, ph, bg, g, gbar, dz, ss);
}

template <typename R>
void launch_adj_update(const Layout& L, R* fbar, R* dbar, const R* gbar, double alpha, double beta, int mode,
                       int klo, int khi, const StepState* ss, cudaStream_t st) {
  adj_update_kernel<R><<<152 * 8, 256, 0, st>>>(L, fbar, dbar, gbar, (R)alpha, (R)beta, mode, klo, khi, ss);
}

template <typename R>
void launch_bz_plane(int nx, int ny, int nz, int k, double dx, double dy, const R* st_in, R* out, int adjoint,
                     const R* bbar, R* lam, cudaStream_t st) {
  const int n = nx * ny;
  bz_plane_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(nx, ny, nz, k, (R)(1.0 / dx), (R)(1.0 / dy), st_in, out, adjoint,
                                                      bbar, lam);
}

#define INST(R)                                                                                                    \
  template void launch_adj_point<R>(const Layout&, const Phys<R>&, const Background<R>&, const R*, const R*, R*,     \
                                    double*, const R*, const R*, const StepState*, int, cudaStream_t);             \
  template void launch_adj_gather<R>(const Layout&, const Phys<R>&, const R*, const R*, R*, const StepState*,       \
                                     cudaStream_t);                                                               \
  template void launch_adj_bc<R>(const Layout&, const Phys<R>&, const Background<R>&, const R*, R*, R,             \
                                 const StepState*, cudaStream_t);                                                 \
  template void launch_adj_update<R>(const Layout&, R*, R*, const R*, double, double, int, int, int,              \
                                     const StepState*, cudaStream_t);                                             \
  template void launch_bz_plane<R>(int, int, int, int, double, double, const R*, R*, int, const R*, R*,             \
                                   cudaStream_t);                                                                 \
  template void launch_adj_pack<R>(const Layout&, int, const R*, R*, cudaStream_t);                                \
  template void launch_adj_unpack<R>(const Layout&, const R*, R*, cudaStream_t);                                   \
  template void launch_d2r<R>(const double*, R*, long long, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mhd

namespace mhd {

// ===========================================================================
// Tiled gather: a block owns 32 x 8 columns and 8 consecutive z points of
// the output (z in [-3, nz+3)) for one group of adjoint fields ({A, ln rho}
// or {u, ln T}); it walks that group's 20 coefficient fields, staging each
// on the block's points plus a 3-cell halo in shared memory (periodic in x
// and y, zero outside the interior layers), and accumulates the transposed
// stencils into 4 targets x 8 z points held in registers.  z stencils reuse
// a 14-value column per thread.  Before it, gd_fold_kernel moves the
// in-plane mixed derivatives into first-derivative coefficients.
// In-plane part of the gradient-of-divergence transpose, folded into the
// first-derivative coefficients before the tiled gather: the mixed term
// (D1_a D1_c)^T G_a = D1_c^T (D1_a^T G_a) for a in {x, y}, so T_a = D1_a^T G_a
// is added to the coefficient of D1_c of component c (c != a).  T_a vanishes
// outside the interior layers (an in-plane stencil of a field that does), so
// nothing is lost at the z ghost layers; the z-direction mixed terms stay in
// the gather.
template <typename R>
__global__ void __launch_bounds__(256) gd_fold_kernel(int nx, int ny, int nz, R* __restrict__ coef, R idx, R idy,
                                                      const StepState* ss) {
  // each thread: E consecutive x points (one 16-byte vector; nx % 4 == 0)
  using V = typename Vec16<R>::T;
  constexpr int E = Vec16<R>::N;
  constexpr int NV = (E + 8) / E;  // vectors covering x = i0 - 4 .. i0 + E + 3
  if (halted(ss)) return;
  const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * E;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i0 >= nx || j >= ny) return;
  const long long n2 = (long long)nx * ny, n3 = n2 * nz;
  const long long row = (long long)k * n2 + (long long)j * nx;
  const R cw[4] = {R(0), W<R>::c1, W<R>::c2, W<R>::c3};
#pragma unroll
  for (int grp = 0; grp < 2; ++grp) {
    // gd(u) coefficients are the lap(u) ones divided by 3
    const int qg = grp == 0 ? CGA : CLU, qd = grp == 0 ? CDA : CDU;
    const R gs = grp == 0 ? R(1) : R(1.0 / 3.0);
    // T_x = D1x^T gd_x at the thread's points; xs[m + 4] = gd_x at i0 + m
    const R* gx = coef + (long long)qg * n3 + row;
    R xs[NV * E];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      int i = i0 - 4 + v * E;
      i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
      V w = __ldg(reinterpret_cast<const V*>(gx + i));
#pragma unroll
      for (int e = 0; e < E; ++e) xs[v * E + e] = vat<V, R>(w, e);
    }
    R tx[E], ty[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      R t = R(0);
#pragma unroll
      for (int m = 1; m <= 3; ++m) t += cw[m] * (xs[4 + e - m] - xs[4 + e + m]);
      tx[e] = gs * idx * t;
      ty[e] = R(0);
    }
    // T_y = D1y^T gd_y: rows j -+ m at the same x
    const R* gy = coef + (long long)(qg + 1) * n3 + (long long)k * n2 + i0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const int jm = j - m < 0 ? j - m + ny : j - m, jp = j + m >= ny ? j + m - ny : j + m;
      V vm = __ldg(reinterpret_cast<const V*>(gy + (long long)jm * nx));
      V vp = __ldg(reinterpret_cast<const V*>(gy + (long long)jp * nx));
#pragma unroll
      for (int e = 0; e < E; ++e) ty[e] += cw[m] * (vat<V, R>(vm, e) - vat<V, R>(vp, e));
    }
    // D1x of component x <- T_y; D1y of component y <- T_x; D1z of component z <- T_x + T_y
    V* cxx = reinterpret_cast<V*>(coef + (long long)(qd + 0) * n3 + row + i0);
    V* cyy = reinterpret_cast<V*>(coef + (long long)(qd + 4) * n3 + row + i0);
    V* czz = reinterpret_cast<V*>(coef + (long long)(qd + 8) * n3 + row + i0);
    V vx = *cxx, vy = *cyy, vz = *czz;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const R yy = gs * idy * ty[e];
      vat<V, R>(vx, e) += yy;
      vat<V, R>(vy, e) += tx[e];
      vat<V, R>(vz, e) += tx[e] + yy;
    }
    *cxx = vx;
    *cyy = vy;
    *czz = vz;
  }
}

namespace gtile {

constexpr int TX = 32, TY = 8, TZ = 8;
// tile rows start 4 columns left of the block (16-byte aligned chunks);
// the block's own columns sit at XO .. XO + 31
constexpr int XO = 4;
constexpr int SX = TX + 8, SY = TY + 6, SZ = TZ + 6;
constexpr int TILE = SX * SY * SZ;

template <typename R>
struct GArgs {
  Layout L;
  Phys<R> ph;
  const R* coef;
  R* dbar;
  R* gbar;
  R* fbar;
  R alpha, beta;     // the substep's update, applied here on layers klo <= k < khi
  int klo, khi;
  const StepState* ss;
  int ntx, nty, ntz;
};

// asynchronous 16-byte copy global -> shared; src_bytes = 0 zero-fills
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 16-byte chunks per tile: chunk c covers tile elements c*EPC .. c*EPC+EPC-1
template <typename R>
__host__ __device__ constexpr int n_chunks() { return TILE * (int)sizeof(R) / 16; }

template <typename R>
__host__ __device__ constexpr size_t smem_bytes(int nbuf) {
  return nbuf * TILE * sizeof(R) + n_chunks<R>() * sizeof(int);
}

// Stage one coefficient field (base: its [nz][ny][nx] array) into s; chunk
// c comes from base + choff[c] (-1: outside the interior layers, zero fill).
template <typename R>
__device__ __forceinline__ void stage_async(R* __restrict__ s, const R* __restrict__ base, const int* choff) {
  constexpr int EPC = 16 / (int)sizeof(R);
  for (int c = threadIdx.y * TX + threadIdx.x; c < n_chunks<R>(); c += TX * TY) {
    const int o = choff[c];
    cp_async16(s + c * EPC, base + (o < 0 ? 0 : o), o < 0 ? 0 : 16);
  }
}

// Stage kinds: what the transposed operator of a coefficient field is, and
// which adjoint field(s) of the block's group it feeds (target t: 0..2
// vector components, 3 the scalar).
//   K_LAP: D2x + D2y + D2z, one axis optionally weighted 4/3 (w: 0 none,
//          1 x, 2 y, 3 z);
//   K_LZ:  D2z, or the weighted Laplacian when w != 0, into component t + 2,
//          and the xz, yz mixed terms (scaled by 1/3 when g is set) into
//          components t and t + 1.
// Gradient-of-divergence terms (gd_a = sum_c D1_a D1_c X_c, D1_a D1_a ->
// D2_a): their in-plane mixed parts are folded into the D1 coefficients
// beforehand (gd_fold_kernel), so gd_x and gd_y take D2 along their own axis
// only (K_D2X, K_D2Y) and gd_z feeds all three components (K_LZ).  For u the
// gd coefficient is the lap(u) coefficient / 3: one staged field serves both,
// with the own-axis D2 weighted 1 + 1/3.
enum { K_VAL = 0, K_D1X, K_D1Y, K_D1Z, K_LAP, K_D2X, K_D2Y, K_LZ };
#define GS(q, kind, t, w, g) ((q) | ((kind) << 8) | ((t) << 12) | ((w) << 16) | ((g) << 18))
// group 0: A and ln rho; group 1: u and ln T
constexpr int NSTAGE_HALF = 20;
__constant__ int kStageHalf[2][NSTAGE_HALF] = {
    {GS(CDA + 0, K_D1X, 0, 0, 0), GS(CDA + 1, K_D1Y, 0, 0, 0), GS(CDA + 2, K_D1Z, 0, 0, 0), GS(CLA + 0, K_LAP, 0, 0, 0),
     GS(CDA + 3, K_D1X, 1, 0, 0), GS(CDA + 4, K_D1Y, 1, 0, 0), GS(CDA + 5, K_D1Z, 1, 0, 0), GS(CLA + 1, K_LAP, 1, 0, 0),
     GS(CDA + 6, K_D1X, 2, 0, 0), GS(CDA + 7, K_D1Y, 2, 0, 0), GS(CDA + 8, K_D1Z, 2, 0, 0), GS(CLA + 2, K_LAP, 2, 0, 0),
     GS(CGA + 0, K_D2X, 0, 0, 0), GS(CGA + 1, K_D2Y, 1, 0, 0), GS(CGA + 2, K_LZ, 0, 0, 0),
     GS(CV + LR, K_VAL, 3, 0, 0), GS(CGL + 0, K_D1X, 3, 0, 0), GS(CGL + 1, K_D1Y, 3, 0, 0), GS(CGL + 2, K_D1Z, 3, 0, 0),
     GS(CLL, K_LAP, 3, 0, 0)},
    {GS(CV + UX, K_VAL, 0, 0, 0), GS(CDU + 0, K_D1X, 0, 0, 0), GS(CDU + 1, K_D1Y, 0, 0, 0), GS(CDU + 2, K_D1Z, 0, 0, 0),
     GS(CLU + 0, K_LAP, 0, 1, 0),
     GS(CV + UY, K_VAL, 1, 0, 0), GS(CDU + 3, K_D1X, 1, 0, 0), GS(CDU + 4, K_D1Y, 1, 0, 0), GS(CDU + 5, K_D1Z, 1, 0, 0),
     GS(CLU + 1, K_LAP, 1, 2, 0),
     GS(CV + UZ, K_VAL, 2, 0, 0), GS(CDU + 6, K_D1X, 2, 0, 0), GS(CDU + 7, K_D1Y, 2, 0, 0), GS(CDU + 8, K_D1Z, 2, 0, 0),
     GS(CLU + 2, K_LZ, 0, 3, 1),
     GS(CV + LT, K_VAL, 3, 0, 0), GS(CGT + 0, K_D1X, 3, 0, 0), GS(CGT + 1, K_D1Y, 3, 0, 0), GS(CGT + 2, K_D1Z, 3, 0, 0),
     GS(CLT, K_LAP, 3, 0, 0)}};
#undef GS

// index of staged point (x offset dx, y offset dy, z point zz + dz) of the
// thread's column
__device__ __forceinline__ int sidx(int tx, int ty, int zz, int dx, int dy, int dz) {
  return ((zz + 3 + dz) * SY + (ty + 3 + dy)) * SX + (tx + XO + dx);
}

// Transposed 1D stencils along x or y (AXIS 0 / 1) at the TZ points of the
// thread's column: D1^T = -D1, D2^T = D2
template <typename R, int AXIS>
__device__ __forceinline__ void t_d1_xy(const R* s, R (&r)[TZ], int tx, int ty, R inv) {
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    R v = R(0);
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const R cm = m == 1 ? W<R>::c1 : (m == 2 ? W<R>::c2 : W<R>::c3);
      const int dx = AXIS == 0 ? m : 0, dy = AXIS == 1 ? m : 0;
      v += cm * (s[sidx(tx, ty, zz, -dx, -dy, 0)] - s[sidx(tx, ty, zz, dx, dy, 0)]);
    }
    r[zz] += v * inv;
  }
}
template <typename R, int AXIS>
__device__ __forceinline__ void t_d2_xy(const R* s, R (&r)[TZ], int tx, int ty, R inv2) {
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    R v = W<R>::e0 * s[sidx(tx, ty, zz, 0, 0, 0)];
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const R em = m == 1 ? W<R>::e1 : (m == 2 ? W<R>::e2 : W<R>::e3);
      const int dx = AXIS == 0 ? m : 0, dy = AXIS == 1 ? m : 0;
      v += em * (s[sidx(tx, ty, zz, -dx, -dy, 0)] + s[sidx(tx, ty, zz, dx, dy, 0)]);
    }
    r[zz] += v * inv2;
  }
}
// the thread's column (z points -3 .. TZ+2) at x, y offsets dx, dy
template <typename R>
__device__ __forceinline__ void load_col(const R* s, R (&col)[SZ], int tx, int ty, int dx, int dy) {
#pragma unroll
  for (int z = 0; z < SZ; ++z) col[z] = s[(z * SY + ty + 3 + dy) * SX + tx + XO + dx];
}
template <typename R>
__device__ __forceinline__ void t_d1_z(const R (&col)[SZ], R (&r)[TZ], R inv) {
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz)
    r[zz] += inv * (W<R>::c1 * (col[zz + 2] - col[zz + 4]) + W<R>::c2 * (col[zz + 1] - col[zz + 5]) +
                    W<R>::c3 * (col[zz] - col[zz + 6]));
}
template <typename R>
__device__ __forceinline__ void t_d2_z(const R (&col)[SZ], R (&r)[TZ], R inv2) {
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz)
    r[zz] += inv2 * (W<R>::e0 * col[zz + 3] + W<R>::e1 * (col[zz + 2] + col[zz + 4]) +
                     W<R>::e2 * (col[zz + 1] + col[zz + 5]) + W<R>::e3 * (col[zz] + col[zz + 6]));
}
// mixed D1h D1z, h = x or y: D1h of the staged columns, then D1z
template <typename R, int AXIS>
__device__ __forceinline__ void t_mix_hz(const R* s, R (&r)[TZ], int tx, int ty, R ihz) {
  R h[SZ];
#pragma unroll
  for (int z = 0; z < SZ; ++z) h[z] = R(0);
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    const R cm = m == 1 ? W<R>::c1 : (m == 2 ? W<R>::c2 : W<R>::c3);
    const int dx = AXIS == 0 ? m : 0, dy = AXIS == 1 ? m : 0;
#pragma unroll
    for (int z = 0; z < SZ; ++z)
      h[z] += cm * (s[(z * SY + ty + 3 + dy) * SX + tx + XO + dx] - s[(z * SY + ty + 3 - dy) * SX + tx + XO - dx]);
  }
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz)
    r[zz] += ihz * (W<R>::c1 * (h[zz + 4] - h[zz + 2]) + W<R>::c2 * (h[zz + 5] - h[zz + 1]) +
                    W<R>::c3 * (h[zz + 6] - h[zz]));
}

// acc[f] += r with a runtime field index (each case indexes registers)
template <typename R, int NO>
__device__ __forceinline__ void add_to(R (&acc)[NO][TZ], int f, const R (&r)[TZ]) {
  switch (f) {
#define ADDF(F)                                                                  \
  case F:                                                                        \
    if (F < NO) {                                                                \
      _Pragma("unroll") for (int zz = 0; zz < TZ; ++zz) acc[F < NO ? F : 0][zz] += r[zz]; \
    }                                                                            \
    break;
    ADDF(0) ADDF(1) ADDF(2) ADDF(3) ADDF(4) ADDF(5) ADDF(6) ADDF(7)
#undef ADDF
    default: break;
  }
}

// Output of one thread's column: on layers klo <= k < khi the substep's
// update F += G, D = alpha D + beta F (loads of a pair of z points issued
// before their stores: fb, db, gb do not alias); elsewhere G (with the
// nudging value adjoints, Eqs. 4 and 5: A_x, A_y at the photosphere and the
// stateful u_x, u_y ghost rows below it) into gbar.
template <typename R, int NO>
__device__ __forceinline__ void epilogue_rows(const Layout& L, const Phys<R>& ph, R* __restrict__ fb,
                                              R* __restrict__ db, R* __restrict__ gb, R alpha, R beta, R dt,
                                              int klo, int khi, const R (&acc)[NO][TZ], int grp, int z0, int j,
                                              int i) {
#pragma unroll
  for (int z2 = 0; z2 < TZ; z2 += 2) {
    R fo[2][NO], dd[2][NO];
    long long qq[2][NO];
    bool fz[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = z0 + z2 + h;
      fz[h] = k >= klo && k < khi;
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        const int f = grp == 0 ? (l < 3 ? AX + l : LR) : (l < 3 ? UX + l : LT);
        qq[h][l] = L.at(f, k, j, i);
        fo[h][l] = fz[h] ? fb[qq[h][l]] : R(0);
        dd[h][l] = (fz[h] || (ph.bcz == 0 && k <= 0)) ? db[qq[h][l]] : R(0);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = z0 + z2 + h;
      if (k >= L.nz + NG) break;
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        const int f = grp == 0 ? (l < 3 ? AX + l : LR) : (l < 3 ? UX + l : LT);
        const R v = acc[l][z2 + h];
        if (fz[h]) {
          const R fv = fo[h][l] + v;
          fb[qq[h][l]] = fv;
          db[qq[h][l]] = alpha * dd[h][l] + beta * fv;
        } else {
          R g = v;
          if (ph.bcz == 0 && ((k == 0 && (f == AX || f == AY)) || (k < 0 && (f == UX || f == UY))))
            g -= (f == AX || f == AY ? ph.tau_A : ph.tau_u) * dt * dd[h][l];
          gb[qq[h][l]] = g;
        }
      }
    }
  }
}

template <typename R, int NO>
__device__ __forceinline__ void epilogue(const GArgs<R>& a, const R (&acc)[NO][TZ], int grp, int z0, int j, int i) {
  epilogue_rows<R, NO>(a.L, a.ph, a.fbar, a.dbar, a.gbar, a.alpha, a.beta, R(a.ss->dt), a.klo, a.khi, acc, grp, z0,
                       j, i);
}

// Each block owns one output group (blockIdx.x & 1: {A, ln rho} or {u, ln T})
// of a tile; NB staging buffers give a prefetch distance of NB - 1 stages.
template <typename R, int NB, int MINB>
__global__ void __launch_bounds__(256, MINB) gather_tiled_kernel(GArgs<R> a) {
  constexpr int NO = 4;  // output fields per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sb = reinterpret_cast<R*>(smem_raw);
  int* choff = reinterpret_cast<int*>(sb + NB * TILE);
  const Layout& L = a.L;
  if (halted(a.ss)) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int grp = (int)(blockIdx.x & 1);
  const int blk = (int)(blockIdx.x >> 1);
  const int* stab = kStageHalf[grp];
  constexpr int NST = NSTAGE_HALF;
  const int bz = blk % a.ntz, bxy = blk / a.ntz;
  const int x0 = (bxy % a.ntx) * TX, y0 = (bxy / a.ntx) * TY, z0 = bz * TZ - NG;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long n3 = (long long)nx * ny * nz;
  {
    constexpr int EPC = 16 / (int)sizeof(R), CH = SX / EPC;
    for (int c = ty * TX + tx; c < n_chunks<R>(); c += TX * TY) {
      const int r = c / CH, ch = c - r * CH;
      const int yy = r % SY, zz = r / SY;
      const int j = ((y0 - 3 + yy) % ny + ny) % ny, k = z0 - 3 + zz;
      const int i = ((x0 - XO + ch * EPC) % nx + nx) % nx;
      choff[c] = (k >= 0 && k < nz) ? (k * ny + j) * nx + i : -1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB - 1; ++b) {
    stage_async<R>(sb + b * TILE, a.coef + (long long)(stab[b] & 255) * n3, choff);
    cp_async_commit();
  }
  const Phys<R>& ph = a.ph;
  R acc[NO][TZ];
#pragma unroll
  for (int f = 0; f < NO; ++f)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) acc[f][zz] = R(0);

#pragma unroll 1
  for (int st = 0; st < NST; ++st) {
    // wait for this stage's field (with NB = 3 the one prefetched after it
    // may still be in flight), make it visible, then prefetch NB - 1 stages
    // ahead into the buffer every thread finished with in the previous stage
    if (NB == 3 && st + 1 < NST) cp_async_wait<1>(); else cp_async_wait<0>();
    __syncthreads();
    const R* s = sb + (st % NB) * TILE;
    if (st + NB - 1 < NST) {
      stage_async<R>(sb + ((st + NB - 1) % NB) * TILE, a.coef + (long long)(stab[st + NB - 1] & 255) * n3, choff);
      cp_async_commit();
    }
    const int code = stab[st];
    const int kind = (code >> 8) & 15, f = (code >> 12) & 15, w = (code >> 16) & 3;
    R r0[TZ];
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) r0[zz] = R(0);
    if (kind == K_VAL) {
#pragma unroll
      for (int zz = 0; zz < TZ; ++zz) r0[zz] = s[sidx(tx, ty, zz, 0, 0, 0)];
      add_to(acc, f, r0);
    } else if (kind == K_D1X) {
      t_d1_xy<R, 0>(s, r0, tx, ty, ph.idx);
      add_to(acc, f, r0);
    } else if (kind == K_D1Y) {
      t_d1_xy<R, 1>(s, r0, tx, ty, ph.idy);
      add_to(acc, f, r0);
    } else if (kind == K_D1Z) {
      R col[SZ];
      load_col(s, col, tx, ty, 0, 0);
      t_d1_z<R>(col, r0, ph.idz);
      add_to(acc, f, r0);
    } else if (kind == K_D2X) {
      t_d2_xy<R, 0>(s, r0, tx, ty, ph.idx2);
      add_to(acc, f, r0);
    } else if (kind == K_D2Y) {
      t_d2_xy<R, 1>(s, r0, tx, ty, ph.idy2);
      add_to(acc, f, r0);
    } else {
      // K_LAP, K_LZ: weighted Laplacian (or D2z alone for gd_z of A)
      const int tgt = kind == K_LAP ? f : f + 2;
      const R four3 = R(4.0 / 3.0);
      if (kind == K_LAP || w != 0) {
        t_d2_xy<R, 0>(s, r0, tx, ty, (w == 1 ? four3 : R(1)) * ph.idx2);
        t_d2_xy<R, 1>(s, r0, tx, ty, (w == 2 ? four3 : R(1)) * ph.idy2);
      }
      {
        R col[SZ];
        load_col(s, col, tx, ty, 0, 0);
        t_d2_z<R>(col, r0, (w == 3 ? four3 : R(1)) * ph.idz2);
      }
      add_to(acc, tgt, r0);
      if (kind == K_LZ) {
        const R g = (code >> 18) & 1 ? R(1.0 / 3.0) : R(1);
#pragma unroll
        for (int zz = 0; zz < TZ; ++zz) r0[zz] = R(0);
        t_mix_hz<R, 0>(s, r0, tx, ty, g * ph.idx * ph.idz);
        add_to(acc, f, r0);
#pragma unroll
        for (int zz = 0; zz < TZ; ++zz) r0[zz] = R(0);
        t_mix_hz<R, 1>(s, r0, tx, ty, g * ph.idy * ph.idz);
        add_to(acc, f + 1, r0);
      }
    }
  }

  const int i = x0 + tx, j = y0 + ty;
  if (i >= nx || j >= ny) return;
  epilogue<R, NO>(a, acc, grp, z0, j, i);
}

}  // namespace gtile

// chunk offsets are 32-bit; rows must split into 16-byte chunks
bool adj_gather_tiled_ok(const Layout& L) { return (long long)L.nx * L.ny * L.nz < (1LL << 31) && L.nx % 4 == 0; }

template <typename R>
void launch_adj_gather_tiled(const Layout& L, const Phys<R>& ph, R* coef, R* dbar, R* gbar, R* fbar, double alpha,
                             double beta, int klo, int khi, const StepState* ss, cudaStream_t st) {
  {
    constexpr int E = Vec16<R>::N;
    const int tpx = L.nx / E;                       // threads per row
    const int bx = tpx < 64 ? tpx : 64, by = 256 / bx;
    gd_fold_kernel<R><<<dim3((tpx + bx - 1) / bx, (L.ny + by - 1) / by, L.nz), dim3(bx, by), 0, st>>>(
        L.nx, L.ny, L.nz, coef, ph.idx, ph.idy, ss);
  }
  gtile::GArgs<R> a;
  a.L = L; a.ph = ph; a.coef = coef; a.dbar = dbar; a.gbar = gbar; a.ss = ss;
  a.fbar = fbar; a.alpha = (R)alpha; a.beta = (R)beta; a.klo = klo; a.khi = khi;
  a.ntx = (L.nx + gtile::TX - 1) / gtile::TX;
  a.nty = (L.ny + gtile::TY - 1) / gtile::TY;
  a.ntz = (L.nz + 2 * NG + gtile::TZ - 1) / gtile::TZ;
  const int nblk = a.ntx * a.nty * a.ntz;
  const dim3 blk(gtile::TX, gtile::TY);
  constexpr int NB = 2;
  const size_t smem = gtile::smem_bytes<R>(NB);
  auto k = gtile::gather_tiled_kernel<R, NB, sizeof(R) == 4 ? 3 : 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<2 * nblk, blk, smem, st>>>(a);
}

template void launch_adj_gather_tiled<float>(const Layout&, const Phys<float>&, float*, float*, float*, float*,
                                             double, double, int, int, const StepState*, cudaStream_t);
template void launch_adj_gather_tiled<double>(const Layout&, const Phys<double>&, double*, double*, double*,
                                              double*, double, double, int, int, const StepState*, cudaStream_t);

}  // namespace mhd
