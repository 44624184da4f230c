// mhd_common.cuh -- layout, parameters and pointwise physics shared by the
// CUDA kernels of libmhd.  (Independent of the CPU oracle: nothing here is
// shared with it.)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

constexpr int NG = 3;     // ghost layers per side (Sect. 2.4, 2.5)
constexpr int XOFF = 8;   // interior x = 0 sits at element 8 of a padded row:
                          // rows (pitch a multiple of 8 elements) start on
                          // 32-byte sectors, so a warp's row of interior cells
                          // is whole sectors, and tile loads starting 4 cells
                          // left of an interior multiple of 4 are 16-byte
                          // aligned (TMA)
constexpr int NF = 8;
enum Field { AX = 0, AY, AZ, UX, UY, UZ, LR, LT };

// Padded SoA layout [field][k + 3][j + 3][XOFF + i], row pitch mx elements.
struct Layout {
  int nx, ny, nz;
  int mx, my, mz;
  long long fs;  // elements per field (multiple of 64)
  __host__ __device__ __forceinline__ long long at(int f, int k, int j, int i) const {
    return (long long)f * fs + ((long long)(k + NG) * my + (j + NG)) * mx + (i + XOFF);
  }
  __host__ __device__ __forceinline__ long long sy() const { return mx; }
  __host__ __device__ __forceinline__ long long sz() const { return (long long)my * mx; }
};

inline Layout make_layout(int nx, int ny, int nz) {
  Layout L;
  L.nx = nx; L.ny = ny; L.nz = nz;
  // x from -XOFF to the last periodic image (nx + 3, written by the pair
  // kernels), rounded to whole 32-byte sectors
  L.mx = (XOFF + nx + 4 + 7) / 8 * 8;
  L.my = ny + 2 * NG;
  L.mz = nz + 2 * NG;
  long long n = (long long)L.mx * L.my * L.mz;
  L.fs = (n + 63) / 64 * 64;
  return L;
}

// Scheme constants in the arithmetic type R.
template <typename R>
struct Phys {
  R idx, idy, idz;        // inverse spacings
  R idx2, idy2, idz2;     // inverse squared spacings
  R gamma, gm1, gz;
  R nu, eta, kappa0, drho;
  R eta_s, chi_s, drho_s;
  R tau_u, tau_A;
  R bext[3];
  int bcz;
  // Newtonian cooling (Sect. 3.1): rate, density cut-off (e-folds below the
  // photospheric value, transition width), height cut-off (z_max, width),
  // layer spacing; the term acts on layers k < nc_k1 (c_z > 0 there)
  R nc_tau, nc_lmag, nc_lw, nc_zmax, nc_zw, dz;
  int nc_k1;
};

// ln rho and ln T are stored as perturbations about fixed background
// profiles (the initial stratification rho0(z), T0(z)); by linearity of the
// stencils the discrete equations are unchanged, but FP32 storage then carries
// rounding relative to the perturbation instead of to |ln rho| ~ 10, which
// otherwise shows up as spurious hydrostatic forces T grad ln rho.  The
// background and its sixth-order z derivatives are computed in FP64 on the
// host.
template <typename R>
struct Background {
  const R* lbar;   // [nz + 6] ln rho background, index k + 3
  const R* tbar;   // [nz + 6] ln T background
  const R* dl;     // [nz] D1_z lbar at interior layers
  const R* d2l;    // [nz] D2_z lbar
  const R* dt;     // [nz] D1_z tbar
  const R* d2t;    // [nz] D2_z tbar
  R cb[4];         // bottom ghost rule constants, index m = 1..3
  R ctT[4];        // top ln T rule constants
  R ctL[4];        // top ln rho rule constants
  // A stored as a perturbation A' about a fixed field A_bg (params
  // a_background; all null otherwise).  The stencils are linear, so
  // B = curl A' + bB, J = grad div A' - lap A' + bJ, and on the swamp layers
  // lap A = lap A' + bL[0..2], div A = div A' + bL[3]; these tables come from
  // FP64 stencils of the ghost-filled A_bg.
  const R* bB;     // [3][nz][ny][nx] curl A_bg
  const R* bJ;     // [3][nz][ny][nx] grad div A_bg - lap A_bg
  const R* bL;     // [4][nz - ksw][ny][nx] lap A_bg (3), div A_bg on layers k >= ksw
  const R* abg;    // A_bg itself in the padded layout, fields 0..2 (read, write)
  int ksw;         // first layer with a nonzero swamp weight or slope
  // Non-uniform vertical grid (params z; all null on the uniform grid): per
  // interior layer dxi/dz, (d2xi/dz2) / (dxi/dz) (so that
  // D_z^2 f = m1^2 D_xi^2 f + r21 D_z f), the position and the cell extent
  // (z_{k+1} - z_{k-1}) / 2.  The ghost rules take dzb[m] = z_{1-m} - z_{-m}
  // below the photosphere and dzt[m] = z_{nz-1+m} - z_{nz-1-m} at the top (on
  // the uniform grid dz and 2 m dz).
  const R* zm1;
  const R* zr21;
  const R* zk;
  const R* zcell;
  R dzb[4];
  R dzt[4];
};

// Device-resident bookkeeping of the time integration (FP64).
struct StepState {
  double t;          // time of the current state
  double dt;         // time step of the current / last step
  double tsub[3];    // substep times t + c_s dt
  double r[3];       // switch-on ramp at tsub
  double s[3];       // driver interpolation weight at tsub
  double stats[8];   // e_kin, e_mag, e_th, mass, flux_net, flux_abs, divb_max, spare
  double stats_t;    // time of the diagnostics
  double eval_r, eval_s;   // driver weights of a single RHS evaluation
  double probe_dt;         // time step computed without advancing time
  long long step;
  int nonfinite;
  int items;         // work-item counter of the z-march launches (zeroed before each)
};

// Low-storage RK3 of Williamson (1980): alpha, beta, c per substep.
__host__ __device__ __forceinline__ double rk_alpha(int s) {
  return s == 0 ? 0.0 : (s == 1 ? -5.0 / 9.0 : -153.0 / 128.0);
}
__host__ __device__ __forceinline__ double rk_beta(int s) {
  return s == 0 ? 1.0 / 3.0 : (s == 1 ? 15.0 / 16.0 : 8.0 / 15.0);
}
__host__ __device__ __forceinline__ double rk_c(int s) {
  return s == 0 ? 0.0 : (s == 1 ? 1.0 / 3.0 : 3.0 / 4.0);
}

template <typename R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ float rexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }
template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return sqrt(x); }

template <typename R> __device__ __forceinline__ R rcos(R x);
template <> __device__ __forceinline__ float rcos<float>(float x) { return cosf(x); }
template <> __device__ __forceinline__ double rcos<double>(double x) { return cos(x); }
template <typename R> __device__ __forceinline__ R rsin(R x);
template <> __device__ __forceinline__ float rsin<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double rsin<double>(double x) { return sin(x); }

// Cosine step: 1 for x <= x1 - w, 0 for x >= x1, 0.5 (1 + cos(pi (x - x1 +
// w) / w)) between; *d (if non-null) receives its derivative.
template <typename R>
__device__ __forceinline__ R nc_step(R x, R x1, R w, R* d) {
  if (d) *d = R(0);
  if (x <= x1 - w) return R(1);
  if (x >= x1) return R(0);
  const R pw = R(3.14159265358979323846) / w;
  const R a = pw * (x - x1 + w);
  if (d) *d = R(-0.5) * pw * rsin<R>(a);
  return R(0.5) * (R(1) + rcos<R>(a));
}

// Newtonian cooling (Sect. 3.1, Eqs. 9-10, read as a relaxation of ln T):
// the d ln T/dt term -tau (1 - T*/T) c_rho c_z at layer k for the full
// ln rho = L and ln T = Th, with T* = sqrt(T0(z) T'(rho)) and T'(rho) = T0(z')
// where the initial ln rho profile (bg.lbar, falling with height) equals L,
// by the piecewise-linear inverse over the interior layers (clamped at the
// end layers).  c_rho cuts off nc_lmag e-folds below the photospheric
// density, c_z above nc_zmax, each through a cosine step.  With dTh, dL
// non-null, also the derivatives of the term (for the adjoint).
template <typename R>
__device__ __forceinline__ R nc_term(const Phys<R>& ph, const Background<R>& bg, int nz, int k, R L, R Th, R* dTh,
                                     R* dL) {
  const R* lr = bg.lbar + NG;
  const R* lt = bg.tbar + NG;
  R dcr = R(0);
  const R cz = nc_step<R>(bg.zk ? bg.zk[k] : R(k) * ph.dz, ph.nc_zmax, ph.nc_zw, nullptr);
  const R cr = nc_step<R>(lr[0] - L, ph.nc_lmag, ph.nc_lw, dL ? &dcr : nullptr);
  R lnTp, slope = R(0);
  if (L >= lr[0]) {
    lnTp = lt[0];
  } else if (L <= lr[nz - 1]) {
    lnTp = lt[nz - 1];
  } else {
    int lo = 0, hi = nz - 1;  // lr[lo] >= L > lr[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (lr[mid] >= L) lo = mid; else hi = mid;
    }
    const R s = (L - lr[lo]) / (lr[hi] - lr[lo]);
    lnTp = lt[lo] + s * (lt[hi] - lt[lo]);
    slope = (lt[hi] - lt[lo]) / (lr[hi] - lr[lo]);
  }
  const R r = rexp<R>(R(0.5) * (lt[k] + lnTp) - Th);  // T*/T
  const R c = cr * cz;
  if (dTh) *dTh = -ph.nc_tau * c * r;
  // d/dL: T*/T through ln T'(L); c_rho through its argument lr[0] - L
  if (dL) *dL = -ph.nc_tau * cz * (-r * R(0.5) * slope * cr - (R(1) - r) * dcr);
  return -ph.nc_tau * (R(1) - r) * c;
}


// Sixth-order centred stencil weights.
template <typename R> struct W {
  static constexpr R c1 = R(45.0 / 60.0), c2 = R(-9.0 / 60.0), c3 = R(1.0 / 60.0);
  static constexpr R e0 = R(-490.0 / 180.0), e1 = R(270.0 / 180.0),
                     e2 = R(-27.0 / 180.0), e3 = R(2.0 / 180.0);
};

// First derivative at p along stride s (times inverse spacing).
template <typename R>
__device__ __forceinline__ R d1(const R* __restrict__ p, long long s, R inv) {
  return (W<R>::c1 * (__ldg(p + s) - __ldg(p - s)) + W<R>::c2 * (__ldg(p + 2 * s) - __ldg(p - 2 * s)) +
          W<R>::c3 * (__ldg(p + 3 * s) - __ldg(p - 3 * s))) * inv;
}
template <typename R>
__device__ __forceinline__ R d2(const R* __restrict__ p, long long s, R inv2) {
  return (W<R>::e0 * __ldg(p) + W<R>::e1 * (__ldg(p + s) + __ldg(p - s)) +
          W<R>::e2 * (__ldg(p + 2 * s) + __ldg(p - 2 * s)) + W<R>::e3 * (__ldg(p + 3 * s) + __ldg(p - 3 * s))) * inv2;
}
// Mixed derivative D1_a(D1_b f), written as the product stencil: the sum
// over m, n = 1..3 of c_m c_n [f(+m,+n) - f(+m,-n) - f(-m,+n) + f(-m,-n)]
// (m along sa, n along sb), times ia ib.  Same operator as applying D1_b and
// then D1_a, with 4 operations per (m, n) instead of recomputing six inner
// first derivatives.
template <typename R>
__device__ __forceinline__ R d11(const R* __restrict__ p, long long sa, long long sb, R ia, R ib) {
  const R c[3] = {W<R>::c1, W<R>::c2, W<R>::c3};
  R acc = R(0);
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    R in = R(0);
#pragma unroll
    for (int n = 1; n <= 3; ++n) {
      const R t = (__ldg(p + m * sa + n * sb) - __ldg(p + m * sa - n * sb)) -
                  (__ldg(p - m * sa + n * sb) - __ldg(p - m * sa - n * sb));
      in += c[n - 1] * t;
    }
    acc += c[m - 1] * in;
  }
  return acc * (ia * ib);
}

// Everything the right-hand side needs at one cell.
template <typename R>
struct Cell {
  R A[3], U[3], L, Th;       // values (ln rho, ln T)
  R dA[3][3], dU[3][3];      // dA[c][a] = d_a A_c
  R lapA[3], lapU[3];        // Laplacians
  R gdA[3], gdU[3];          // grad(div .)
  R gL[3], gT[3], lapL, lapT;
};

// Right-hand side of the four evolution equations at one cell
// (ln-variable resistive MHD, mu0 = 1, p = rho T, Weyl gauge):
//  dA/dt  = u x B - eta J + eta_s w lap A + e_z eta_s w' div A        (Eq. 18)
//  du/dt  = -(u.grad)u - T grad(ln rho + ln T) + g_z e_z + J x B / rho
//           + nu (lap u + grad div u / 3 + 2 S.grad ln rho)
//  dlnrho = -u.grad ln rho - div u + D_rho (lap ln rho + |grad ln rho|^2)
//           + chi_rho w lap ln rho                                      (Eq. 20)
//  dlnT   = -u.grad ln T - (gamma-1) div u + (gamma-1)(eta J^2/(rho T) + 2 nu S^2/T)
//           + (gamma-1) kappa0 T^{5/2}/rho (lap ln T + 3.5 |grad ln T|^2)
//           + chi_s w lap ln T                                          (Eq. 19)
// B = curl A + B_ext (Eq. 6), J = grad div A - lap A.  The swamp diffusivity
// is left out of the Ohmic heating (Sect. 4.3.1).  Boundary rows and nudging
// are applied by the caller.
//
// rhs_point_bj takes A's contribution as three vectors -- B = curl A + B_ext,
// J = grad div A - lap A and the swamp part of the induction equation
// sw = eta_s w lap A + eta_s w' div A z^ -- so that a pass that sees only A
// (split right-hand side) can form them; rhs_point forms them from the cell.
template <typename R>
__device__ __forceinline__ void rhs_point_bj(const Cell<R>& c, const Phys<R>& ph, R w, const R B[3], const R J[3],
                                             const R sw[3], R out[8]) {
  const R B0 = B[0], B1 = B[1], B2 = B[2];
  const R J0 = J[0], J1 = J[1], J2 = J[2];
  const R divU = c.dU[0][0] + c.dU[1][1] + c.dU[2][2];
  const R T = rexp<R>(c.Th);
  const R rho1 = rexp<R>(-c.L);
  const R u0 = c.U[0], u1 = c.U[1], u2 = c.U[2];

  // induction
  out[0] = u1 * B2 - u2 * B1 - ph.eta * J0 + sw[0];
  out[1] = u2 * B0 - u0 * B2 - ph.eta * J1 + sw[1];
  out[2] = u0 * B1 - u1 * B0 - ph.eta * J2 + sw[2];

  // traceless rate of strain S_ab = (d_a u_b + d_b u_a)/2 - delta_ab div u / 3
  const R third = R(1.0 / 3.0);
  const R s00 = c.dU[0][0] - third * divU, s11 = c.dU[1][1] - third * divU,
          s22 = c.dU[2][2] - third * divU;
  const R s01 = R(0.5) * (c.dU[0][1] + c.dU[1][0]);
  const R s02 = R(0.5) * (c.dU[0][2] + c.dU[2][0]);
  const R s12 = R(0.5) * (c.dU[1][2] + c.dU[2][1]);
  const R S2 = s00 * s00 + s11 * s11 + s22 * s22 + R(2) * (s01 * s01 + s02 * s02 + s12 * s12);
  const R gL0 = c.gL[0], gL1 = c.gL[1], gL2 = c.gL[2];
  const R SgL0 = s00 * gL0 + s01 * gL1 + s02 * gL2;
  const R SgL1 = s01 * gL0 + s11 * gL1 + s12 * gL2;
  const R SgL2 = s02 * gL0 + s12 * gL1 + s22 * gL2;
  // Lorentz force
  const R F0 = J1 * B2 - J2 * B1, F1 = J2 * B0 - J0 * B2, F2 = J0 * B1 - J1 * B0;
  // momentum: dU[c][a] = d_a u_c
  const R adv0 = u0 * c.dU[0][0] + u1 * c.dU[0][1] + u2 * c.dU[0][2];
  const R adv1 = u0 * c.dU[1][0] + u1 * c.dU[1][1] + u2 * c.dU[1][2];
  const R adv2 = u0 * c.dU[2][0] + u1 * c.dU[2][1] + u2 * c.dU[2][2];
  out[3] = -adv0 - T * (gL0 + c.gT[0]) + F0 * rho1 + ph.nu * (c.lapU[0] + third * c.gdU[0] + R(2) * SgL0);
  out[4] = -adv1 - T * (gL1 + c.gT[1]) + F1 * rho1 + ph.nu * (c.lapU[1] + third * c.gdU[1] + R(2) * SgL1);
  out[5] = -adv2 - T * (gL2 + c.gT[2]) + F2 * rho1 + ph.nu * (c.lapU[2] + third * c.gdU[2] + R(2) * SgL2) + ph.gz;

  // continuity
  const R ugL = u0 * gL0 + u1 * gL1 + u2 * gL2;
  const R gL2s = gL0 * gL0 + gL1 * gL1 + gL2 * gL2;
  out[6] = -ugL - divU + ph.drho * (c.lapL + gL2s) + ph.drho_s * w * c.lapL;

  // energy (ln T)
  const R ugT = u0 * c.gT[0] + u1 * c.gT[1] + u2 * c.gT[2];
  const R gT2 = c.gT[0] * c.gT[0] + c.gT[1] * c.gT[1] + c.gT[2] * c.gT[2];
  const R JJ = J0 * J0 + J1 * J1 + J2 * J2;
  const R T1 = R(1) / T;
  const R heat = ph.gm1 * (ph.eta * JJ * rho1 + R(2) * ph.nu * S2) * T1;
  const R kt = ph.gm1 * ph.kappa0 * rexp<R>(R(2.5) * c.Th - c.L);
  out[7] = -ugT - ph.gm1 * divU + heat + kt * (c.lapT + R(3.5) * gT2) + ph.chi_s * w * c.lapT;
}

// B, J and the swamp terms of the induction equation from A's derivatives
template <typename R>
__device__ __forceinline__ void a_terms(const Cell<R>& c, const Phys<R>& ph, R w, R wp, R B[3], R J[3], R sw[3]) {
  B[0] = c.dA[2][1] - c.dA[1][2] + ph.bext[0];
  B[1] = c.dA[0][2] - c.dA[2][0] + ph.bext[1];
  B[2] = c.dA[1][0] - c.dA[0][1] + ph.bext[2];
  J[0] = c.gdA[0] - c.lapA[0];
  J[1] = c.gdA[1] - c.lapA[1];
  J[2] = c.gdA[2] - c.lapA[2];
  const R ews = ph.eta_s * w;
  const R divA = c.dA[0][0] + c.dA[1][1] + c.dA[2][2];
  sw[0] = ews * c.lapA[0];
  sw[1] = ews * c.lapA[1];
  sw[2] = ews * c.lapA[2] + ph.eta_s * wp * divA;
}

template <typename R>
__device__ __forceinline__ void rhs_point(const Cell<R>& c, const Phys<R>& ph, R w, R wp, R out[8]) {
  R B[3], J[3], sw[3];
  a_terms<R>(c, ph, w, wp, B, J, sw);
  rhs_point_bj<R>(c, ph, w, B, J, sw, out);
}

// Error flag checked by every kernel (set by the reductions on NaN/Inf).
__device__ __forceinline__ bool halted(const StepState* ss) {
  return *((volatile const int*)&ss->nonfinite) != 0;
}

}  // namespace mhd
