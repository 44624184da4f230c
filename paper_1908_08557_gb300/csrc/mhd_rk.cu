// mhd_rk.cu -- fused right-hand side + low-storage RK3 update.
//
// One thread per interior cell.  Substep s of the Williamson (1980) 2N
// scheme: df <- alpha_s df + dt RHS(f_in, t_s); f_out <- f_in + beta_s df.
// Substep 0 does not read df (alpha = 0), substep 2 does not write it.
// The new value is also stored into the periodic x,y images of the cell, so
// the next substep finds its rims filled.  Photospheric threads (k = 0) also
// advance the stateful u_x, u_y ghost layers below the photosphere, which
// carry only the nudging term of Eq. 5.
#include "mhd_internal.h"

namespace mhd {

template <typename R>
struct RKArgs {
  Layout L;
  Phys<R> ph;
  Background<R> bg;
  const R* fin;
  R* fout;
  R* df;
  const R* wtab;
  const R* wptab;
  const R* axt;
  const R* ayt;
  const R* v0;
  const R* v1;
  const StepState* ss;
  int sub;
};

// store v at (k, j, i) and at its periodic x,y images inside the padded plane
template <typename R>
__device__ __forceinline__ void store_images(const Layout& L, R* __restrict__ f, int fl, int k, int j, int i, R v) {
  int xs[3], ys[3], nxs = 1, nys = 1;
  xs[0] = i;
  ys[0] = j;
  if (i < NG) xs[nxs++] = i + L.nx;
  if (i >= L.nx - NG) xs[nxs++] = i - L.nx;
  if (j < NG) ys[nys++] = j + L.ny;
  if (j >= L.ny - NG) ys[nys++] = j - L.ny;
  for (int b = 0; b < nys; ++b)
    for (int a = 0; a < nxs; ++a) f[L.at(fl, k, ys[b], xs[a])] = v;
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 2 : 0) rk_simple_kernel(RKArgs<R> a) {
  const Layout& L = a.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  if (halted(a.ss)) return;
  const Phys<R>& ph = a.ph;
  const long long st[3] = {1, L.sy(), L.sz()};
  // a non-uniform vertical grid: z derivatives scaled by dxi/dz of the layer,
  // and D_z^2 f = (dxi/dz)^2 D_xi^2 f + r21 D_z f (added below)
  const bool zg = a.bg.zm1 != nullptr;
  const R m1 = zg ? a.bg.zm1[k] : ph.idz, r21 = zg ? a.bg.zr21[k] : R(0);
  const R inv[3] = {ph.idx, ph.idy, m1};
  const R inv2[3] = {ph.idx2, ph.idy2, zg ? m1 * m1 : ph.idz2};
  const R* base[NF];
#pragma unroll
  for (int fl = 0; fl < NF; ++fl) base[fl] = a.fin + L.at(fl, k, j, i);

  Cell<R> c;
  R a2[3], u2[3];  // own-axis second derivatives d_c^2 A_c, d_c^2 u_c (Laplacian and grad div share them)
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    const R* pa = base[AX + cc];
    const R* pu = base[UX + cc];
    c.A[cc] = *pa;
    c.U[cc] = *pu;
    c.lapA[cc] = R(0);
    c.lapU[cc] = R(0);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      c.dA[cc][ax] = d1(pa, st[ax], inv[ax]);
      c.dU[cc][ax] = d1(pu, st[ax], inv[ax]);
      R da2 = d2(pa, st[ax], inv2[ax]), du2 = d2(pu, st[ax], inv2[ax]);
      if (ax == 2 && zg) {
        da2 += r21 * c.dA[cc][2];
        du2 += r21 * c.dU[cc][2];
      }
      if (ax == cc) {
        a2[cc] = da2;
        u2[cc] = du2;
      }
      c.lapA[cc] += da2;
      c.lapU[cc] += du2;
    }
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    R sa = R(0), su = R(0);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      if (cc == ax) {
        sa += a2[cc];
        su += u2[cc];
      } else {
        sa += d11(base[AX + cc], st[ax], st[cc], inv[ax], inv[cc]);
        su += d11(base[UX + cc], st[ax], st[cc], inv[ax], inv[cc]);
      }
    }
    c.gdA[ax] = sa;
    c.gdU[ax] = su;
  }
  // ln rho, ln T: stored perturbation + background (value and FP64-built
  // z derivatives of the background)
  c.L = a.bg.lbar[k + NG] + *base[LR];
  c.Th = a.bg.tbar[k + NG] + *base[LT];
  c.lapL = R(0);
  c.lapT = R(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    c.gL[ax] = d1(base[LR], st[ax], inv[ax]);
    c.gT[ax] = d1(base[LT], st[ax], inv[ax]);
    c.lapL += d2(base[LR], st[ax], inv2[ax]);
    c.lapT += d2(base[LT], st[ax], inv2[ax]);
  }
  if (zg) {
    c.lapL += r21 * c.gL[2];
    c.lapT += r21 * c.gT[2];
  }
  c.gL[2] += a.bg.dl[k];
  c.lapL += a.bg.d2l[k];
  c.gT[2] += a.bg.dt[k];
  c.lapT += a.bg.d2t[k];
  R out[NF];
  {
    const R w = a.wtab[k], wp = a.wptab[k];
    R B[3], J[3], sw[3];
    a_terms<R>(c, ph, w, wp, B, J, sw);
    if (a.bg.bB) {
      // A stored about a background: add its B, J and (swamp layers) its
      // lap A, div A terms, all linear in A
      const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
      const long long q3 = (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        B[cc] += a.bg.bB[cc * n3 + q3];
        J[cc] += a.bg.bJ[cc * n3 + q3];
      }
      if (k >= a.bg.ksw) {
        const long long ns = n2 * (L.nz - a.bg.ksw), qs = (long long)(k - a.bg.ksw) * n2 + (long long)j * L.nx + i;
        const R ews = ph.eta_s * w;
        sw[0] += ews * a.bg.bL[qs];
        sw[1] += ews * a.bg.bL[ns + qs];
        sw[2] += ews * a.bg.bL[2 * ns + qs] + ph.eta_s * wp * a.bg.bL[3 * ns + qs];
      }
    }
    rhs_point_bj<R>(c, ph, w, B, J, sw, out);
  }
  if (k < ph.nc_k1) out[LT] += nc_term<R>(ph, a.bg, L.nz, k, c.L, c.Th, nullptr, nullptr);

  // substep constants
  const int sub = a.sub;
  const bool eval = sub < 0;
  const R dt = eval ? R(1) : R(a.ss->dt);
  const R alpha = eval ? R(0) : R(rk_alpha(sub));
  const R beta = eval ? R(0) : R(rk_beta(sub));
  R tgx = R(0), tgy = R(0);
  if (ph.bcz == 0 && k == 0) {
    const double r = eval ? a.ss->eval_r : a.ss->r[sub];
    const double s = eval ? a.ss->eval_s : a.ss->s[sub];
    const long long q2 = (long long)j * L.nx + i, n2 = (long long)L.nx * L.ny;
    const R vx = a.v0[q2] + R(s) * (a.v1[q2] - a.v0[q2]);
    const R vy = a.v0[n2 + q2] + R(s) * (a.v1[n2 + q2] - a.v0[n2 + q2]);
    tgx = R(r) * vx;
    tgy = R(r) * vy;
    // photospheric rows: nudging of A_hor (Sect. 2.1) and u_hor (Eq. 5);
    // ln rho held at its initial profile and u_z = 0 (Sect. 2.5)
    out[AX] -= ph.tau_A * (c.A[0] - a.axt[q2]);
    out[AY] -= ph.tau_A * (c.A[1] - a.ayt[q2]);
    out[UX] -= ph.tau_u * (c.U[0] - tgx);
    out[UY] -= ph.tau_u * (c.U[1] - tgy);
    out[UZ] = R(0);
    out[LR] = R(0);
  }
  if (ph.bcz == 0 && k == L.nz - 1) out[UZ] = R(0);  // closed top (Sect. 4)

#pragma unroll
  for (int fl = 0; fl < NF; ++fl) {
    const long long q = L.at(fl, k, j, i);
    const R dfn = (sub > 0 ? alpha * a.df[q] : R(0)) + dt * out[fl];
    if (sub < 2) a.df[q] = dfn;
    if (!eval) store_images<R>(L, a.fout, fl, k, j, i, a.fin[q] + beta * dfn);
  }
  if (ph.bcz == 0 && k == 0) {
    for (int m = 1; m <= NG; ++m) {
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const long long q = L.at(UX + cc, -m, j, i);
        const R u = a.fin[q];
        const R rh = -ph.tau_u * (u - (cc == 0 ? tgx : tgy));
        const R dfn = (sub > 0 ? alpha * a.df[q] : R(0)) + dt * rh;
        if (sub < 2) a.df[q] = dfn;
        if (!eval) store_images<R>(L, a.fout, UX + cc, -m, j, i, u + beta * dfn);
      }
    }
  }
}

template <typename R>
void launch_rk(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* fin, R* fout, R* df,
               const R* wtab, const R* wptab, const Driver& drv, const StepState* ss, int sub, cudaStream_t st) {
  RKArgs<R> a;
  a.L = L;
  a.ph = ph;
  a.bg = bg;
  a.fin = fin;
  a.fout = fout;
  a.df = df;
  a.wtab = wtab;
  a.wptab = wptab;
  a.axt = (const R*)drv.axt;
  a.ayt = (const R*)drv.ayt;
  a.v0 = (const R*)drv.v0;
  a.v1 = (const R*)drv.v1;
  a.ss = ss;
  a.sub = sub;
  dim3 blk(32, 8, 1);
  dim3 grd((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
  rk_simple_kernel<R><<<grd, blk, 0, st>>>(a);
}

template void launch_rk<float>(const Layout&, const Phys<float>&, const Background<float>&, const float*,
                               float*, float*, const float*, const float*, const Driver&, const StepState*, int,
                               cudaStream_t);
template void launch_rk<double>(const Layout&, const Phys<double>&, const Background<double>&, const double*,
                                double*, double*, const double*, const double*, const Driver&,
                                const StepState*, int, cudaStream_t);

}  // namespace mhd
