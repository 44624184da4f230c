// mhd_adjoint_point.cuh -- the pointwise part of the adjoint of the
// right-hand side (transpose of rhs_point and of the photospheric rows),
// shared by the one-thread-per-cell adjoint kernel and the TMA-fed z-march
// kernel.
#pragma once
#include "mhd_common.cuh"

namespace mhd {

// Coefficient indices: the adjoints of the cell-record entries the
// right-hand side reads.  Two entries need no field of their own:
//  - the values of A enter only through the photospheric nudging (Eq. 4),
//    whose adjoint the gather applies from D directly;
//  - gd(u) enters only through the viscous force nu (lap u + gd(u) / 3), so
//    its adjoint is the lap(u) coefficient divided by 3.
enum {
  CV = -UX,      // value adjoints of u_x, u_y, u_z, ln rho, ln T at CV + field
  CDA = 5,       // dA[c][a] at CDA + 3c + a
  CDU = 14,      // dU[c][a]
  CLA = 23,      // lapA[c]
  CLU = 26,      // lapU[c] (3 gdU[c] is the same number)
  CGA = 29,      // gdA[a]
  CGL = 32,      // gL[a]
  CGT = 35,      // gT[a]
  CLL = 38,      // lapL
  CLT = 39,      // lapT
  NCOEF = 40
};

// Transpose of rhs_point (see mhd_common.cuh) at one cell: given the output
// adjoint w[8], accumulate the adjoints of every input of the cell record.
// Forward intermediates are recomputed in the same order.
template <typename R>
__device__ __forceinline__ void rhs_point_adjoint(const Cell<R>& c, const Phys<R>& ph, R w_, R wp, const R wo[8],
                                                  R cf[NCOEF]) {
  for (int q = 0; q < NCOEF; ++q) cf[q] = R(0);
  // forward
  const R B0 = c.dA[2][1] - c.dA[1][2] + ph.bext[0];
  const R B1 = c.dA[0][2] - c.dA[2][0] + ph.bext[1];
  const R B2 = c.dA[1][0] - c.dA[0][1] + ph.bext[2];
  const R J0 = c.gdA[0] - c.lapA[0], J1 = c.gdA[1] - c.lapA[1], J2 = c.gdA[2] - c.lapA[2];
  const R divU = c.dU[0][0] + c.dU[1][1] + c.dU[2][2];
  const R T = rexp<R>(c.Th);
  const R rho1 = rexp<R>(-c.L);
  const R u0 = c.U[0], u1 = c.U[1], u2 = c.U[2];
  const R third = R(1.0 / 3.0);
  const R s00 = c.dU[0][0] - third * divU, s11 = c.dU[1][1] - third * divU, s22 = c.dU[2][2] - third * divU;
  const R s01 = R(0.5) * (c.dU[0][1] + c.dU[1][0]);
  const R s02 = R(0.5) * (c.dU[0][2] + c.dU[2][0]);
  const R s12 = R(0.5) * (c.dU[1][2] + c.dU[2][1]);
  const R S2 = s00 * s00 + s11 * s11 + s22 * s22 + R(2) * (s01 * s01 + s02 * s02 + s12 * s12);
  const R gL0 = c.gL[0], gL1 = c.gL[1], gL2 = c.gL[2];
  const R F0 = J1 * B2 - J2 * B1, F1 = J2 * B0 - J0 * B2, F2 = J0 * B1 - J1 * B0;
  const R JJ = J0 * J0 + J1 * J1 + J2 * J2;
  const R T1 = R(1) / T;
  const R Q = ph.eta * JJ * rho1 + R(2) * ph.nu * S2;
  const R kt = ph.gm1 * ph.kappa0 * rexp<R>(R(2.5) * c.Th - c.L);
  const R gT2 = c.gT[0] * c.gT[0] + c.gT[1] * c.gT[1] + c.gT[2] * c.gT[2];

  R bB0 = 0, bB1 = 0, bB2 = 0, bJ0 = 0, bJ1 = 0, bJ2 = 0, bu0 = 0, bu1 = 0, bu2 = 0;
  R bdivA = 0, bdivU = 0, bT = 0, brho1 = 0, bTh = 0, bL = 0;
  R bs00 = 0, bs11 = 0, bs22 = 0, bs01 = 0, bs02 = 0, bs12 = 0;
  R bF0 = 0, bF1 = 0, bF2 = 0, bS2 = 0;
  R bgL0 = 0, bgL1 = 0, bgL2 = 0;

  // induction
  {
    const R a0 = wo[0], a1 = wo[1], a2 = wo[2];
    const R ews = ph.eta_s * w_;
    bu1 += a0 * B2; bB2 += a0 * u1; bu2 -= a0 * B1; bB1 -= a0 * u2; bJ0 -= ph.eta * a0; cf[CLA + 0] += ews * a0;
    bu2 += a1 * B0; bB0 += a1 * u2; bu0 -= a1 * B2; bB2 -= a1 * u0; bJ1 -= ph.eta * a1; cf[CLA + 1] += ews * a1;
    bu0 += a2 * B1; bB1 += a2 * u0; bu1 -= a2 * B0; bB0 -= a2 * u1; bJ2 -= ph.eta * a2; cf[CLA + 2] += ews * a2;
    bdivA += ph.eta_s * wp * a2;
  }
  // momentum
  const R Fc[3] = {F0, F1, F2};
  R bFc[3] = {0, 0, 0};
  R bSgL[3] = {0, 0, 0};
  for (int cc = 0; cc < 3; ++cc) {
    const R a = wo[3 + cc];
    // -(u.grad) u_c
    bu0 -= a * c.dU[cc][0];
    bu1 -= a * c.dU[cc][1];
    bu2 -= a * c.dU[cc][2];
    cf[CDU + 3 * cc + 0] -= a * u0;
    cf[CDU + 3 * cc + 1] -= a * u1;
    cf[CDU + 3 * cc + 2] -= a * u2;
    // -T (gL + gT)
    bT -= a * (c.gL[cc] + c.gT[cc]);
    if (cc == 0) bgL0 -= a * T;
    if (cc == 1) bgL1 -= a * T;
    if (cc == 2) bgL2 -= a * T;
    cf[CGT + cc] -= a * T;
    // F / rho
    bFc[cc] += a * rho1;
    brho1 += a * Fc[cc];
    // viscous force
    cf[CLU + cc] += ph.nu * a;  // and nu / 3 for gd(u)_c: implied (see the enum)
    bSgL[cc] += R(2) * ph.nu * a;
  }
  bF0 = bFc[0]; bF1 = bFc[1]; bF2 = bFc[2];
  // Lorentz force
  bJ1 += bF0 * B2; bB2 += bF0 * J1; bJ2 -= bF0 * B1; bB1 -= bF0 * J2;
  bJ2 += bF1 * B0; bB0 += bF1 * J2; bJ0 -= bF1 * B2; bB2 -= bF1 * J0;
  bJ0 += bF2 * B1; bB1 += bF2 * J0; bJ1 -= bF2 * B0; bB0 -= bF2 * J1;
  // S . grad ln rho
  bs00 += bSgL[0] * gL0; bs01 += bSgL[0] * gL1; bs02 += bSgL[0] * gL2;
  bgL0 += bSgL[0] * s00; bgL1 += bSgL[0] * s01; bgL2 += bSgL[0] * s02;
  bs01 += bSgL[1] * gL0; bs11 += bSgL[1] * gL1; bs12 += bSgL[1] * gL2;
  bgL0 += bSgL[1] * s01; bgL1 += bSgL[1] * s11; bgL2 += bSgL[1] * s12;
  bs02 += bSgL[2] * gL0; bs12 += bSgL[2] * gL1; bs22 += bSgL[2] * gL2;
  bgL0 += bSgL[2] * s02; bgL1 += bSgL[2] * s12; bgL2 += bSgL[2] * s22;
  // continuity
  {
    const R a = wo[6];
    bu0 -= a * gL0; bu1 -= a * gL1; bu2 -= a * gL2;
    bgL0 -= a * u0; bgL1 -= a * u1; bgL2 -= a * u2;
    bdivU -= a;
    cf[CLL] += a * (ph.drho + ph.drho_s * w_);
    bgL0 += a * ph.drho * R(2) * gL0;
    bgL1 += a * ph.drho * R(2) * gL1;
    bgL2 += a * ph.drho * R(2) * gL2;
  }
  // energy
  {
    const R a = wo[7];
    bu0 -= a * c.gT[0]; bu1 -= a * c.gT[1]; bu2 -= a * c.gT[2];
    cf[CGT + 0] -= a * u0; cf[CGT + 1] -= a * u1; cf[CGT + 2] -= a * u2;
    bdivU -= a * ph.gm1;
    // heat = gm1 Q T1
    const R bQ = a * ph.gm1 * T1;
    const R bT1 = a * ph.gm1 * Q;
    const R bJJ = bQ * ph.eta * rho1;
    brho1 += bQ * ph.eta * JJ;
    bS2 += bQ * R(2) * ph.nu;
    bJ0 += R(2) * J0 * bJJ; bJ1 += R(2) * J1 * bJJ; bJ2 += R(2) * J2 * bJJ;
    bT -= bT1 * T1 * T1;
    // conduction kt (lapT + 3.5 gT2) and swamp
    const R bkt = a * (c.lapT + R(3.5) * gT2);
    cf[CLT] += a * kt + a * ph.chi_s * w_;
    cf[CGT + 0] += a * kt * R(7) * c.gT[0];
    cf[CGT + 1] += a * kt * R(7) * c.gT[1];
    cf[CGT + 2] += a * kt * R(7) * c.gT[2];
    bTh += bkt * kt * R(2.5);
    bL -= bkt * kt;
  }
  // S2
  bs00 += R(2) * s00 * bS2; bs11 += R(2) * s11 * bS2; bs22 += R(2) * s22 * bS2;
  bs01 += R(4) * s01 * bS2; bs02 += R(4) * s02 * bS2; bs12 += R(4) * s12 * bS2;
  // strain components
  cf[CDU + 0] += bs00; cf[CDU + 4] += bs11; cf[CDU + 8] += bs22;
  bdivU -= third * (bs00 + bs11 + bs22);
  cf[CDU + 1] += R(0.5) * bs01; cf[CDU + 3] += R(0.5) * bs01;
  cf[CDU + 2] += R(0.5) * bs02; cf[CDU + 6] += R(0.5) * bs02;
  cf[CDU + 5] += R(0.5) * bs12; cf[CDU + 7] += R(0.5) * bs12;
  // exponentials
  bTh += bT * T;
  bL -= brho1 * rho1;
  // divergences
  cf[CDU + 0] += bdivU; cf[CDU + 4] += bdivU; cf[CDU + 8] += bdivU;
  cf[CDA + 0] += bdivA; cf[CDA + 4] += bdivA; cf[CDA + 8] += bdivA;
  // J = gdA - lapA
  cf[CGA + 0] += bJ0; cf[CGA + 1] += bJ1; cf[CGA + 2] += bJ2;
  cf[CLA + 0] -= bJ0; cf[CLA + 1] -= bJ1; cf[CLA + 2] -= bJ2;
  // B = curl A
  cf[CDA + 3 * 2 + 1] += bB0; cf[CDA + 3 * 1 + 2] -= bB0;
  cf[CDA + 3 * 0 + 2] += bB1; cf[CDA + 3 * 2 + 0] -= bB1;
  cf[CDA + 3 * 1 + 0] += bB2; cf[CDA + 3 * 0 + 1] -= bB2;
  // values and first derivatives of ln rho
  cf[CV + UX] += bu0; cf[CV + UY] += bu1; cf[CV + UZ] += bu2;
  cf[CV + LR] += bL; cf[CV + LT] += bTh;
  cf[CGL + 0] += bgL0; cf[CGL + 1] += bgL1; cf[CGL + 2] += bgL2;
}

// Adjoint of one interior cell's right-hand-side row in substep `sub`.  wo
// holds dt * D at the cell on entry (D: adjoint of the RK accumulator); rows
// the boundary overwrites carry no dependence and are masked; the nudging
// terms (Eqs. 4 and 5) give value adjoints and, at the photosphere, the
// driver adjoints accumulated into thbar ([6][ny][nx]: A target x, y; v0
// x, y; v1 x, y).  dux, duy point at D of u_x, u_y at (k = 0, j, i) and sz
// is the z stride: the stateful ghost rows below sit at -m sz.  cf receives
// the NCOEF coefficients; the value adjoint of A_x, A_y from the nudging,
// -tau_A dt D, is left to the gather.
template <typename R>
__device__ __forceinline__ void adjoint_cell(const Cell<R>& c, const Phys<R>& ph, R w_, R wp, R (&wo)[NF], R dt,
                                             int k, int nz, const R* dux, const R* duy, long long sz,
                                             double* thbar, long long q2, long long n2, const StepState* ss, int sub,
                                             R (&cf)[NCOEF]) {
  R vU0 = R(0), vU1 = R(0);
  if (ph.bcz == 0 && k == 0) {
    wo[UZ] = R(0);
    wo[LR] = R(0);
    // nudging: -tau_A (A_hor - A_target), -tau_u (u_hor - r v*)
    vU0 = -ph.tau_u * wo[UX];
    vU1 = -ph.tau_u * wo[UY];
    const double r = ss->r[sub], s = ss->s[sub];
    double tgx = (double)(ph.tau_u * wo[UX]), tgy = (double)(ph.tau_u * wo[UY]);
    // stateful ghost rows below the photosphere: nudging only
    for (int m = 1; m <= NG; ++m) {
      tgx += (double)(ph.tau_u * dt * dux[-m * sz]);
      tgy += (double)(ph.tau_u * dt * duy[-m * sz]);
    }
    thbar[0 * n2 + q2] += (double)(ph.tau_A * wo[AX]);
    thbar[1 * n2 + q2] += (double)(ph.tau_A * wo[AY]);
    thbar[2 * n2 + q2] += r * (1.0 - s) * tgx;
    thbar[3 * n2 + q2] += r * (1.0 - s) * tgy;
    thbar[4 * n2 + q2] += r * s * tgx;
    thbar[5 * n2 + q2] += r * s * tgy;
  }
  if (ph.bcz == 0 && k == nz - 1) wo[UZ] = R(0);
  rhs_point_adjoint<R>(c, ph, w_, wp, wo, cf);
  cf[CV + UX] += vU0;
  cf[CV + UY] += vU1;
}

// Adjoint of the Newtonian cooling term of the ln T equation (Sect. 3.1):
// its derivatives by ln T and ln rho, times the output adjoint of ln T, into
// the value adjoints of the two.
template <typename R>
__device__ __forceinline__ void nc_adjoint(const Phys<R>& ph, const Background<R>& bg, int nz, int k, R L, R Th, R wT,
                                           R (&cf)[NCOEF]) {
  R dTh, dL;
  nc_term<R>(ph, bg, nz, k, L, Th, &dTh, &dL);
  cf[CV + LT] += wT * dTh;
  cf[CV + LR] += wT * dL;
}

}  // namespace mhd
