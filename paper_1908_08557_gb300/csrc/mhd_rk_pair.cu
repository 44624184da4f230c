// mhd_rk_pair.cu -- FP32 right-hand side + RK3 update in one TMA-fed z-march
// pass, two x-adjacent cells per thread in packed f32x2 arithmetic, with the z
// histories of every thread's cells kept in tensor memory (TMEM).
//
// A CTA (128 threads) owns a 32 x 8 tile and marches in z over a chunk of
// layers; thread (tx, ty) owns cells (x0 + 2tx, x0 + 2tx + 1, y0 + ty).
// Plane p of all 8 fields, with its 3-cell halo, arrives in shared memory
// through one 4D cp.async.bulk.tensor load into a 5-slot ring (planes k .. k+3
// in use at centre k, k+4 in flight), guarded by mbarriers with bounded waits.
//
//  front (plane k + 3): each thread copies its two cells of the 8 fields into
//    TMEM (ring of 8 planes) and forms the sources of the xz / yz mixed
//    derivatives -- D1x X_z, D1y X_z, D1x X_x + D1y X_y for X = A, u -- also
//    into a TMEM ring of 8 planes;
//  centre (plane k): D1z and D2z of the fields and D1z of the mixed sources
//    from TMEM (tcgen05.ld), x and y derivatives from the shared ring, the xy
//    mixed derivatives D1x(D1y X_y), D1x(D1y X_x) through a small shared
//    scratch with an x halo (the tensor-product operator D1x D1y equals
//    D1y D1x), the pointwise physics, nudging and boundary rows, the
//    low-storage RK update and the stores (with periodic images).
//
// TMEM: each CTA allocates 256 columns; thread t owns lane t.  Columns
// [0, 128): values, 16 per plane slot (field f, cell c at 2f + c); columns
// [128, 256): mixed sources, 16 per plane slot (source q, cell c at 2q + c).
// The shared ring (> 76 KB per CTA) admits at most two CTAs per SM, so the
// two allocations never exceed the SM's 512 columns and tcgen05.alloc never
// waits.  Every exit path deallocates.
#include <cuda.h>

#include "mhd_adjoint_point.cuh"
#include "mhd_internal.h"
#include "mhd_pair.cuh"
#include "mhd_zmarch.cuh"

namespace mhd {
namespace pair {

using namespace pk;

constexpr int TX = zm::TX, TY = zm::TY;  // 32 x 8 cells
constexpr int BX = zm::BX, BY = zm::BY;  // 40 x 14 box
constexpr int NT = TX / 2 * TY;          // 128 threads
constexpr int NR = 5;                    // shared ring slots
constexpr int FP = BY * BX;              // floats per field plane of a box
constexpr int PLANE = NF * FP;           // floats per ring slot (17920 B)
constexpr int NSC = 4;                   // scratch fields: D1y A_y, D1y A_x, D1y u_y, D1y u_x
constexpr int SCF = TY * BX;             // floats per scratch field
constexpr int DFT = NF * TY * TX;        // floats per RK-accumulator tile (8 KB)
constexpr size_t SMEM_BYTES = (size_t)NR * PLANE * 4 + (size_t)NSC * SCF * 4 + (size_t)2 * DFT * 4 + (NR + 2) * 8 + 16;
static_assert(SMEM_BYTES > 233472 / 3, "ring must keep TMEM users at <= 2 CTAs per SM");
constexpr int TMEM_COLS = 256;
constexpr int VCOL = 0, SCOL = 128;      // value / source rings in TMEM

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
  Coef cx, cy, cz;
  // adjoint mode: D (adjoint of the RK accumulator, padded layout; the
  // accumulator tiles then carry D), the NCOEF coefficient fields
  // ([NCOEF][nz][ny][nx]) and the driver adjoints out
  const float* dbar;
  float* coef;
  double* thbar;
  // bounded waits: polls before a ring or accumulator wait gives up; and a
  // test hook for the time-out path: the CTA that takes work item 0 does
  // not issue the copy of plane skip_plane in it (INT_MIN: every copy is
  // issued), so its wait for that plane runs out with no copy in flight
  int wait_limit;
  int skip_plane;
  // work items claimed from a counter (StepState::items) instead of taken
  // by grid stride
  int dyn;
};

// ---- TMEM access (32x32b shape: each thread its own lane) -----------------
#define TM_R16(a)                                                                                          \
  "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), \
      "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
#define TM_W16(a)                                                                                              \
  "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), \
      "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15])

struct V16 {
  uint32_t r[16];
  __device__ __forceinline__ f2 get(int q) const { return make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1])); }
  __device__ __forceinline__ void set(int q, f2 v) {
    r[2 * q] = __float_as_uint(v.x);
    r[2 * q + 1] = __float_as_uint(v.y);
  }
};
__device__ __forceinline__ void tm_ld(uint32_t t, V16& v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : TM_R16(v.r)
      : "r"(t));
}
__device__ __forceinline__ void tm_st(uint32_t t, const V16& v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(t),
      TM_W16(v.r)
      : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- a packed pair of FP32 numbers with the arithmetic the templated
// pointwise adjoint uses (each operation one f32x2 instruction, or two
// scalar ones for division and exp: the hardware approximations, as in the
// forward mode) -------------------------------------------------------------
struct P2 {
  f2 v;
  __device__ __forceinline__ P2() {}
  __device__ __forceinline__ P2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ P2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ P2(int a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ explicit P2(f2 a) : v(a) {}
  __device__ __forceinline__ P2& operator+=(P2 b) { v = add(v, b.v); return *this; }
  __device__ __forceinline__ P2& operator-=(P2 b) { v = dif(v, b.v); return *this; }
};
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2(add(a.v, b.v)); }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2(dif(a.v, b.v)); }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2(mul(a.v, b.v)); }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(mul(a.v, F2(-1.f))); }
__device__ __forceinline__ P2 operator/(P2 a, P2 b) {
  return P2(make_float2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)));
}
}  // namespace pair
template <> __device__ __forceinline__ pair::P2 rexp<pair::P2>(pair::P2 x) {
  return pair::P2(make_float2(__expf(x.v.x), __expf(x.v.y)));
}
namespace pair {

// ---- adjoint mode: the derivatives the pointwise adjoint reads, then the
// per-cell transpose (adjoint_cell) of each of the pair's two cells --------
__device__ __forceinline__ void adjoint_centre(const Args& a, const float* Pk, const float* Praw, float* scr,
                                               const float* dtile, uint64_t* dbar_mb, uint32_t& dphase,
                                               uint32_t& dpending, int k, int k0, int x0, int y0,
                                               const f2 (&vz)[NF], const f2 (&d1z)[NF], const f2 (&d2z)[NF],
                                               const f2 (&mz)[6], float wk, float wpk, float lbk, float tbk,
                                               float dlk, float dtk, float d2tk, float dt, int sub) {
  const Layout& L = a.L;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, warp = tid >> 5;
  const int e = 2 * tx + 4;
  // y derivatives of A_y, A_x (also the sources of the xy-mixed terms of
  // grad div A) and of u_y, u_x; the scratch holds D1y A_y, D1y A_x on the
  // tile plus an x halo (fields 0, 1; warps 0, 1 compute the halo items)
  f2 dyAy, yyAy, dyAx, yyAx, dyUy, dyUx;
  ds_pair(Pk + AY * FP, BX, a.cy, dyAy, &yyAy);
  ds_pair(Pk + AX * FP, BX, a.cy, dyAx, &yyAx);
  ds_pair(Pk + UY * FP, BX, a.cy, dyUy, nullptr);
  ds_pair(Pk + UX * FP, BX, a.cy, dyUx, nullptr);
  {
    float* sc = scr + ty * BX + e;
    *reinterpret_cast<f2*>(sc + 0 * SCF) = dyAy;
    *reinterpret_cast<f2*>(sc + 1 * SCF) = dyAx;
    if (warp < 2) {
      const int hr = (tid & 31) >> 2, hx = ((tid & 3) < 2) ? 2 * (tid & 3) : 32 + 2 * (tid & 3);
      f2 h;
      ds_pair(Praw + (warp == 0 ? AY : AX) * FP + (hr + 3) * BX + hx, BX, a.cy, h, nullptr);
      *reinterpret_cast<f2*>(scr + warp * SCF + hr * BX + hx) = h;
    }
  }
  __syncthreads();
  f2 m0, m1;
  dx_pair(scr + 0 * SCF + ty * BX + e, a.cx, m0, nullptr);
  dx_pair(scr + 1 * SCF + ty * BX + e, a.cx, m1, nullptr);
  // A: off-diagonal first derivatives, Laplacians, grad div
  f2 dxAy, xxAy, dxAz, xxAz, dyAz, yyAz, dxAx, xxAx;
  dx_pair(Pk + AX * FP, a.cx, dxAx, &xxAx);
  dx_pair(Pk + AY * FP, a.cx, dxAy, &xxAy);
  dx_pair(Pk + AZ * FP, a.cx, dxAz, &xxAz);
  ds_pair(Pk + AZ * FP, BX, a.cy, dyAz, &yyAz);
  const f2 lapA0 = add(add(xxAx, yyAx), d2z[AX]);
  const f2 lapA1 = add(add(xxAy, yyAy), d2z[AY]);
  const f2 lapA2 = add(add(xxAz, yyAz), d2z[AZ]);
  const f2 gdA0 = add(add(xxAx, m0), mz[0]);
  const f2 gdA1 = add(add(m1, yyAy), mz[1]);
  const f2 gdA2 = add(mz[2], d2z[AZ]);
  // u: first derivatives; ln rho, ln T: gradients, Laplacian of ln T
  f2 U00, U10, U20, U21, gL0, gL1, gT0, gT1, xxT, yyT;
  dx_pair(Pk + UX * FP, a.cx, U00, nullptr);
  dx_pair(Pk + UY * FP, a.cx, U10, nullptr);
  dx_pair(Pk + UZ * FP, a.cx, U20, nullptr);
  ds_pair(Pk + UZ * FP, BX, a.cy, U21, nullptr);
  dx_pair(Pk + LR * FP, a.cx, gL0, nullptr);
  ds_pair(Pk + LR * FP, BX, a.cy, gL1, nullptr);
  dx_pair(Pk + LT * FP, a.cx, gT0, &xxT);
  ds_pair(Pk + LT * FP, BX, a.cy, gT1, &yyT);
  const f2 lapT = add(add(add(xxT, yyT), d2z[LT]), F2(d2tk));
  // D of the pair (bounded wait; a time-out is recorded and the CTA goes on)
  const int sl = (k - k0) & 1;
  if (!zm::mbar_wait(dbar_mb, (dphase >> sl) & 1u)) atomicOr(&a.ss->nonfinite, 2);
  dphase ^= 1u << sl;
  if (tid == 0) dpending &= ~(1u << sl);
  f2 dq[NF];
  {
    const float* d = dtile + ty * TX + 2 * tx;
#pragma unroll
    for (int f = 0; f < NF; ++f) dq[f] = ld2(d + f * TY * TX);
  }
  const int i = x0 + 2 * tx, j = y0 + ty;
  if (i >= L.nx || j >= L.ny) return;
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  if (k > 0 || a.ph.bcz != 0) {
    // both cells at once: the templated transpose on packed pairs
    const Phys<float>& pf = a.ph;
    Phys<P2> pp;
    pp.idx = pf.idx; pp.idy = pf.idy; pp.idz = pf.idz;
    pp.idx2 = pf.idx2; pp.idy2 = pf.idy2; pp.idz2 = pf.idz2;
    pp.gamma = pf.gamma; pp.gm1 = pf.gm1; pp.gz = pf.gz;
    pp.nu = pf.nu; pp.eta = pf.eta; pp.kappa0 = pf.kappa0; pp.drho = pf.drho;
    pp.eta_s = pf.eta_s; pp.chi_s = pf.chi_s; pp.drho_s = pf.drho_s;
    pp.tau_u = pf.tau_u; pp.tau_A = pf.tau_A;
    pp.bext[0] = pf.bext[0]; pp.bext[1] = pf.bext[1]; pp.bext[2] = pf.bext[2];
    pp.bcz = pf.bcz;
    Cell<P2> cl;
    cl.A[0] = P2(vz[AX]); cl.A[1] = P2(vz[AY]); cl.A[2] = P2(vz[AZ]);
    cl.U[0] = P2(vz[UX]); cl.U[1] = P2(vz[UY]); cl.U[2] = P2(vz[UZ]);
    cl.L = P2(add(F2(lbk), vz[LR]));
    cl.Th = P2(add(F2(tbk), vz[LT]));
    cl.dA[0][0] = P2(dxAx); cl.dA[0][1] = P2(dyAx); cl.dA[0][2] = P2(d1z[AX]);
    cl.dA[1][0] = P2(dxAy); cl.dA[1][1] = P2(dyAy); cl.dA[1][2] = P2(d1z[AY]);
    cl.dA[2][0] = P2(dxAz); cl.dA[2][1] = P2(dyAz); cl.dA[2][2] = P2(d1z[AZ]);
    cl.dU[0][0] = P2(U00); cl.dU[0][1] = P2(dyUx); cl.dU[0][2] = P2(d1z[UX]);
    cl.dU[1][0] = P2(U10); cl.dU[1][1] = P2(dyUy); cl.dU[1][2] = P2(d1z[UY]);
    cl.dU[2][0] = P2(U20); cl.dU[2][1] = P2(U21); cl.dU[2][2] = P2(d1z[UZ]);
    cl.lapA[0] = P2(lapA0); cl.lapA[1] = P2(lapA1); cl.lapA[2] = P2(lapA2);
    cl.gdA[0] = P2(gdA0); cl.gdA[1] = P2(gdA1); cl.gdA[2] = P2(gdA2);
    // the adjoint reads no second derivative of u and no Laplacian of ln rho
    cl.lapU[0] = cl.lapU[1] = cl.lapU[2] = P2(0.f);
    cl.gdU[0] = cl.gdU[1] = cl.gdU[2] = P2(0.f);
    cl.lapL = P2(0.f);
    cl.gL[0] = P2(gL0); cl.gL[1] = P2(gL1); cl.gL[2] = P2(add(d1z[LR], F2(dlk)));
    cl.gT[0] = P2(gT0); cl.gT[1] = P2(gT1); cl.gT[2] = P2(add(d1z[LT], F2(dtk)));
    cl.lapT = P2(lapT);
    P2 wo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) wo[f] = P2(mul(F2(dt), dq[f]));
    // closed top: du_z/dt = 0 (the photosphere is the scalar path below)
    if (pf.bcz == 0 && k == L.nz - 1) wo[UZ] = P2(0.f);
    P2 cf[NCOEF];
    rhs_point_adjoint<P2>(cl, pp, P2(wk), P2(wpk), wo, cf);
    if (k < pf.nc_k1) {
      // Newtonian cooling, one cell at a time
      float dT0, dL0, dT1, dL1;
      nc_term<float>(pf, a.bg, L.nz, k, cl.L.v.x, cl.Th.v.x, &dT0, &dL0);
      nc_term<float>(pf, a.bg, L.nz, k, cl.L.v.y, cl.Th.v.y, &dT1, &dL1);
      cf[CV + LT] += wo[LT] * P2(make_float2(dT0, dT1));
      cf[CV + LR] += wo[LT] * P2(make_float2(dL0, dL1));
    }
    float* co = a.coef + (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
    for (int q = 0; q < NCOEF; ++q) *reinterpret_cast<f2*>(co + q * n3) = cf[q].v;
    return;
  }
  // photosphere: one cell at a time (nudging rows, FP64 driver adjoints)
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    auto P = [c](f2 v) { return c == 0 ? v.x : v.y; };
    Cell<float> cl;
    cl.A[0] = P(vz[AX]); cl.A[1] = P(vz[AY]); cl.A[2] = P(vz[AZ]);
    cl.U[0] = P(vz[UX]); cl.U[1] = P(vz[UY]); cl.U[2] = P(vz[UZ]);
    cl.L = lbk + P(vz[LR]);
    cl.Th = tbk + P(vz[LT]);
    cl.dA[0][0] = P(dxAx); cl.dA[0][1] = P(dyAx); cl.dA[0][2] = P(d1z[AX]);
    cl.dA[1][0] = P(dxAy); cl.dA[1][1] = P(dyAy); cl.dA[1][2] = P(d1z[AY]);
    cl.dA[2][0] = P(dxAz); cl.dA[2][1] = P(dyAz); cl.dA[2][2] = P(d1z[AZ]);
    cl.dU[0][0] = P(U00); cl.dU[0][1] = P(dyUx); cl.dU[0][2] = P(d1z[UX]);
    cl.dU[1][0] = P(U10); cl.dU[1][1] = P(dyUy); cl.dU[1][2] = P(d1z[UY]);
    cl.dU[2][0] = P(U20); cl.dU[2][1] = P(U21); cl.dU[2][2] = P(d1z[UZ]);
    cl.lapA[0] = P(lapA0); cl.lapA[1] = P(lapA1); cl.lapA[2] = P(lapA2);
    cl.gdA[0] = P(gdA0); cl.gdA[1] = P(gdA1); cl.gdA[2] = P(gdA2);
    // the adjoint reads no second derivative of u and no Laplacian of ln rho
    cl.lapU[0] = cl.lapU[1] = cl.lapU[2] = 0.f;
    cl.gdU[0] = cl.gdU[1] = cl.gdU[2] = 0.f;
    cl.lapL = 0.f;
    cl.gL[0] = P(gL0); cl.gL[1] = P(gL1); cl.gL[2] = P(d1z[LR]) + dlk;
    cl.gT[0] = P(gT0); cl.gT[1] = P(gT1); cl.gT[2] = P(d1z[LT]) + dtk;
    cl.lapT = P(lapT);
    float wo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) wo[f] = dt * P(dq[f]);
    const long long q2 = (long long)j * L.nx + i + c;
    const long long cu = L.at(UX, 0, j, i + c);
    float cf[NCOEF];
    adjoint_cell<float>(cl, a.ph, wk, wpk, wo, dt, k, L.nz, a.dbar + cu, a.dbar + cu + L.fs, L.sz(), a.thbar, q2,
                        n2, a.ss, sub, cf);
    if (k < a.ph.nc_k1) nc_adjoint<float>(a.ph, a.bg, L.nz, k, cl.L, cl.Th, wo[LT], cf);
    float* co = a.coef + (long long)k * n2 + q2;
#pragma unroll
    for (int q = 0; q < NCOEF; ++q) co[q * n3] = cf[q];
  }
}

// ---- the kernel -------------------------------------------------------------
// ADJ = false: right-hand side + RK update of substep `sub` (sub < 0: store
// the right-hand side only).  ADJ = true: the pointwise adjoint of substep
// `sub` (the input is the ghost-filled substep state, tmd maps D): per
// interior cell the NCOEF coefficients of the transposed right-hand side and,
// at the photosphere, the driver adjoints; no state is stored.
// NC: the forward right-hand side includes the Newtonian cooling term (a
// separate instantiation, so that the default path carries none of it).
// BG: A is stored about a background field; the background's B, J (every
// cell) and lap A, div A (swamp layers) come from per-cell tables.
// ZG: a non-uniform vertical grid (the z stencils in index space, the metric
// applied per layer); separate instantiations keep the uniform path as lean
// as before.
template <bool ADJ, bool NC, bool BG, bool ZG>
__global__ void __launch_bounds__(NT, 2) rk_pair_kernel(const __grid_constant__ CUtensorMap tm,
                                                        const __grid_constant__ CUtensorMap tmd, const Args a) {
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;
  float* scr = raw + NR * PLANE;
  float* dfs = scr + NSC * SCF;           // RK accumulator tiles of centres k (double buffer)
  uint64_t* mbar = (uint64_t*)(dfs + 2 * DFT);
  uint64_t* mbd = mbar + NR;
  uint32_t* tslot = (uint32_t*)(mbd + 2);

  const Layout& L = a.L;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, warp = tid >> 5;
  if (halted(a.ss)) return;
  if (tid == 0) {
    for (int s = 0; s < NR; ++s) zm::mbar_init(&mbar[s]);
    zm::mbar_init(&mbd[0]);
    zm::mbar_init(&mbd[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(zm::sa(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);

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
  const int e = 2 * tx + 4;                 // box x of the thread's first cell
  const int cen = (ty + 3) * BX + e;        // box offset of the pair
  // halo item of the xy-mixed scratch: field hq = warp, row hr, box x hx
  const int hq = warp, hr = (tid & 31) >> 2, hx = ((tid & 3) < 2) ? 2 * (tid & 3) : 32 + 2 * (tid & 3);
  const int hfield = hq == 0 ? AY : (hq == 1 ? AX : (hq == 2 ? UY : UX));
  uint32_t phase = 0, pending = 0;        // shared ring: parities, copies in flight (thread 0)
  uint32_t dphase = 0, dpending = 0;      // accumulator tiles: the same
  const int nitems = a.ntx * a.nty * a.nch;
  const long long n2 = (long long)L.nx * L.ny;
  bool bad = false;

  // RK accumulator tile of centre k (sub > 0) into buffer (k - k0) & 1
  auto load_df = [&](int k, int k0, int x0, int y0) {
    const int s = (k - k0) & 1;
    zm::tma_plane(&tmd, dfs + s * DFT, &mbd[s], DFT * 4, x0 + XOFF, y0 + NG, k + NG, 0);
    dpending |= 1u << s;
  };
  // ring slots are tracked incrementally (slot of plane p = (p - pbase) mod NR)
  auto wrap = [](int s) { return s >= NR ? s - NR : s; };
  bool inject = false;  // the time-out test hook applies to this item
  auto load = [&](int p, int s, int x0, int y0) {
    if (inject && p == a.skip_plane) return;
    zm::tma_plane(&tm, raw + s * PLANE, &mbar[s], PLANE * 4, x0 - 4 + XOFF, y0, p + NG, 0);
    pending |= 1u << s;
  };
  // collective bounded wait for plane p; false on time-out (uniform)
  auto wait = [&](int s) -> bool {
    const bool to = !zm::mbar_wait(&mbar[s], (phase >> s) & 1u, a.wait_limit);
    if (__syncthreads_or(to)) return false;
    phase ^= 1u << s;
    pending &= ~(1u << s);
    return true;
  };
  // front of plane p: values and mixed sources of the pair into TMEM
  auto front = [&](int p, int sp) {
    const float* P = raw + sp * PLANE + cen;
    V16 v, s;
#pragma unroll
    for (int f = 0; f < NF; ++f) v.set(f, ld2(P + f * FP));
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int X = g == 0 ? AX : UX;
      f2 zx, zy, xx, yy;
      dx_pair(P + (X + 2) * FP, a.cx, zx, nullptr);
      ds_pair(P + (X + 2) * FP, BX, a.cy, zy, nullptr);
      dx_pair(P + X * FP, a.cx, xx, nullptr);
      ds_pair(P + (X + 1) * FP, BX, a.cy, yy, nullptr);
      s.set(3 * g + 0, zx);
      s.set(3 * g + 1, zy);
      s.set(3 * g + 2, add(xx, yy));
    }
    s.set(6, F2(0.f));
    s.set(7, F2(0.f));
    tm_st(tlane + VCOL + (uint32_t)(p & 7) * 16, v);
    tm_st(tlane + SCOL + (uint32_t)(p & 7) * 16, s);
  };

  // work items (tile, z chunk) by grid stride, or (dyn, for launches with
  // many items per CTA) by a counter: each CTA then takes the next item when
  // it finishes one, so CTAs that meet dearer items (images at the x, y
  // edges, swamp layers) do not hold up the launch.  Thread 0 claims the
  // following item when it starts one; the claim is handed to the CTA at the
  // end-of-item barrier.  Item order: chunk-fastest (all z chunks of a tile
  // in flight together) for the forward launches by grid stride;
  // tile-fastest (the CTAs running together cover whole rows of tiles of one
  // chunk) for the adjoint and for claimed items, where it measured faster.
  __shared__ int s_next;
  if (a.dyn) {
    if (tid == 0) s_next = atomicAdd(&a.ss->items, 1);
    __syncthreads();
  }
  for (int item = a.dyn ? s_next : (int)blockIdx.x; item < nitems && !bad;) {
    int next = 0;
    if (a.dyn && tid == 0) next = atomicAdd(&a.ss->items, 1);
    const int tiles = a.ntx * a.nty;
    const bool tile_fast = ADJ || a.dyn;
    const int ch = tile_fast ? item / tiles : item % a.nch;
    const int tile = tile_fast ? item - ch * tiles : item / a.nch;
    const int x0 = (tile % a.ntx) * TX, y0 = (tile / a.ntx) * TY;
    const int k0 = ch * a.kchunk, k1 = min(L.nz, k0 + a.kchunk);
    const int pbase = k0 - NG, plast = k1 + NG - 1;
    inject = a.skip_plane != INT_MIN && item == 0;
    if (tid == 0) {
      for (int p = pbase; p <= min(pbase + NR - 1, plast); ++p) load(p, p - pbase, x0, y0);
      if (ADJ || sub > 0) load_df(k0, k0, x0, y0);
    }
    // prologue: planes k0-3 .. k0+2; the three below k0 are released at once
    for (int p = pbase; p < k0 + NG && !bad; ++p) {
      const int sp = wrap(p - pbase);
      bad = !wait(sp);
      if (bad) break;
      // every thread is past the front of p - 1; below k0 that was its last use
      if (p > pbase && p - 1 < k0 && tid == 0 && p - 1 + NR <= plast) load(p - 1 + NR, p - 1 - pbase, x0, y0);
      front(p, sp);
    }
    int sk = NG;  // slot of centre k (k0 - pbase = NG < NR)
    for (int k = k0; k < k1 && !bad; ++k, sk = wrap(sk + 1)) {
      const int s3 = wrap(sk + NG);  // slot of plane k + 3
      const int i = x0 + 2 * tx, j = y0 + ty;
      const bool live = i < L.nx && j < L.ny;
      const long long cq = live ? L.at(0, k, j, i) : 0;
      // per-layer tables, fetched before the waits
      const float wk = a.wtab[k], wpk = a.wptab[k];
      const float lbk = a.bg.lbar[k + NG], tbk = a.bg.tbar[k + NG];
      const float dlk = a.bg.dl[k], dtk = a.bg.dt[k], d2lk = a.bg.d2l[k], d2tk = a.bg.d2t[k];
      // non-uniform vertical grid: the z stencils ran in index space; the
      // metric of layer k (dxi/dz, and r21 with D_z^2 = m1^2 D_xi^2 + r21 D_z)
      float zm1k = 1.f, zr21k = 0.f;
      if constexpr (ZG) {
        zm1k = a.bg.zm1[k];
        zr21k = a.bg.zr21[k];
      }
      // background B, J of the pair (A stored about a background), issued
      // before the waits so that their latency overlaps them
      f2 gB[3], gJ[3];
      if constexpr (BG) {
        const long long n3 = n2 * L.nz, q3 = (long long)k * n2 + (long long)j * L.nx + i;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          gB[cc] = live ? __ldg(reinterpret_cast<const float2*>(a.bg.bB + cc * n3 + q3)) : F2(0.f);
          gJ[cc] = live ? __ldg(reinterpret_cast<const float2*>(a.bg.bJ + cc * n3 + q3)) : F2(0.f);
        }
      }
      bad = !wait(s3);
      if (bad) break;
      if (tid == 0) {
        // every thread is past centre k - 1: plane k - 1's slot takes k + 4,
        // and its accumulator buffer the tile of centre k + 1
        if (k > k0 && k - 1 + NR <= plast) load(k - 1 + NR, wrap(sk + NR - 1), x0, y0);
        if ((ADJ || sub > 0) && k + 1 < k1) load_df(k + 1, k0, x0, y0);
      }
      front(k + NG, s3);
      tm_wait_st();

      const float* Pk = raw + sk * PLANE + cen;
      // ---- z derivatives from the TMEM rings --------------------------------
      f2 vz[NF], d1z[NF], d2z[NF], mz[6];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        vz[f] = ld2(Pk + f * FP);
        d1z[f] = F2(0.f);
        d2z[f] = mul(a.cz.e0, vz[f]);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) mz[q] = F2(0.f);
#pragma unroll
      for (int m = 3; m >= 1; --m) {
        const f2 cm = m == 1 ? a.cz.c1 : (m == 2 ? a.cz.c2 : a.cz.c3);
        const f2 em = m == 1 ? a.cz.e1 : (m == 2 ? a.cz.e2 : a.cz.e3);
        V16 vp, vm, sp, sm;
        tm_ld(tlane + VCOL + (uint32_t)((k + m) & 7) * 16, vp);
        tm_ld(tlane + VCOL + (uint32_t)((k - m) & 7) * 16, vm);
        tm_ld(tlane + SCOL + (uint32_t)((k + m) & 7) * 16, sp);
        tm_ld(tlane + SCOL + (uint32_t)((k - m) & 7) * 16, sm);
        tm_wait_ld();
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          d1z[f] = fma2(cm, dif(vp.get(f), vm.get(f)), d1z[f]);
          d2z[f] = fma2(em, add(vp.get(f), vm.get(f)), d2z[f]);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) mz[q] = fma2(cm, dif(sp.get(q), sm.get(q)), mz[q]);
      }
      if constexpr (ZG) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          d1z[f] = mul(F2(zm1k), d1z[f]);
          d2z[f] = fma2(F2(zr21k), d1z[f], mul(F2(zm1k * zm1k), d2z[f]));
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) mz[q] = mul(F2(zm1k), mz[q]);
      }

      // stateful u_x, u_y ghost rows below the photosphere (k = 0): their
      // values are the TMEM copies of planes -1 .. -3 (loaded warp-wide)
      f2 gux[NG], guy[NG];
      if (!ADJ && a.ph.bcz == 0 && k == 0) {
#pragma unroll
        for (int m = 1; m <= NG; ++m) {
          uint32_t g[4];
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                       : "=r"(g[0]), "=r"(g[1]), "=r"(g[2]), "=r"(g[3])
                       : "r"(tlane + VCOL + (uint32_t)((k - m) & 7) * 16 + 2 * UX));
          tm_wait_ld();
          gux[m - 1] = make_float2(__uint_as_float(g[0]), __uint_as_float(g[1]));
          guy[m - 1] = make_float2(__uint_as_float(g[2]), __uint_as_float(g[3]));
        }
      }

      if constexpr (ADJ) {
        adjoint_centre(a, Pk, raw + sk * PLANE, scr, dfs + ((k - k0) & 1) * DFT, &mbd[(k - k0) & 1], dphase,
                       dpending, k, k0, x0, y0, vz, d1z, d2z, mz, wk, wpk, lbk, tbk, dlk, dtk, d2tk, dt, sub);
        continue;
      }
      // ---- x, y derivatives from the shared ring, folded as they come -------
      // (the own-axis second derivatives D2x A_x, D2y A_y cancel in J outside
      // the swamp layers)
      const bool swamp = wk != 0.f || wpk != 0.f;
      // y derivatives of A_y, A_x, u_y, u_x: also the sources of the xy-mixed
      // terms D1x(D1y .), through the scratch with an x halo
      f2 dyAy, dyAx, yyAx, dyUy, yyUy, dyUx, yyUx, yyAy = F2(0.f);
      if (swamp)
        ds_pair(Pk + AY * FP, BX, a.cy, dyAy, &yyAy);
      else
        ds_pair(Pk + AY * FP, BX, a.cy, dyAy, nullptr);
      ds_pair(Pk + AX * FP, BX, a.cy, dyAx, &yyAx);
      ds_pair(Pk + UY * FP, BX, a.cy, dyUy, &yyUy);
      ds_pair(Pk + UX * FP, BX, a.cy, dyUx, &yyUx);
      {
        float* sc = scr + ty * BX + e;
        *reinterpret_cast<f2*>(sc + 0 * SCF) = dyAy;
        *reinterpret_cast<f2*>(sc + 1 * SCF) = dyAx;
        *reinterpret_cast<f2*>(sc + 2 * SCF) = dyUy;
        *reinterpret_cast<f2*>(sc + 3 * SCF) = dyUx;
        f2 h;
        ds_pair(raw + sk * PLANE + hfield * FP + (hr + 3) * BX + hx, BX, a.cy, h, nullptr);
        *reinterpret_cast<f2*>(scr + hq * SCF + hr * BX + hx) = h;
      }
      __syncthreads();
      f2 mxy[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) dx_pair(scr + q * SCF + ty * BX + e, a.cx, mxy[q], nullptr);

      const Phys<float>& ph = a.ph;
      const f2 w = F2(wk), wp = F2(wpk);
      // A: B = curl A + B_ext, J = grad div A - lap A, swamp terms of the
      // induction equation
      f2 B0, B1, B2, J0, J1, J2, sw0 = F2(0.f), sw1 = F2(0.f), sw2 = F2(0.f);
      {
        f2 dxAy, xxAy, dxAz, xxAz, dyAz, yyAz;
        dx_pair(Pk + AY * FP, a.cx, dxAy, &xxAy);
        dx_pair(Pk + AZ * FP, a.cx, dxAz, &xxAz);
        ds_pair(Pk + AZ * FP, BX, a.cy, dyAz, &yyAz);
        B0 = add(dif(dyAz, d1z[AY]), F2(ph.bext[0]));
        B1 = add(dif(d1z[AX], dxAz), F2(ph.bext[1]));
        B2 = add(dif(dxAy, dyAx), F2(ph.bext[2]));
        if (!swamp) {
          J0 = dif(dif(add(mxy[0], mz[0]), yyAx), d2z[AX]);
          J1 = dif(dif(add(mxy[1], mz[1]), xxAy), d2z[AY]);
          J2 = dif(dif(mz[2], xxAz), yyAz);
        } else {
          f2 dxAx, xxAx;
          dx_pair(Pk + AX * FP, a.cx, dxAx, &xxAx);
          const f2 lap0 = add(add(xxAx, yyAx), d2z[AX]);
          const f2 lap1 = add(add(xxAy, yyAy), d2z[AY]);
          const f2 lap2 = add(add(xxAz, yyAz), d2z[AZ]);
          J0 = dif(add(add(xxAx, mxy[0]), mz[0]), lap0);
          J1 = dif(add(add(mxy[1], yyAy), mz[1]), lap1);
          J2 = dif(add(mz[2], d2z[AZ]), lap2);
          const f2 ews = mul(F2(ph.eta_s), w);
          f2 divA = add(add(dxAx, dyAy), d1z[AZ]);
          f2 l0 = lap0, l1 = lap1, l2 = lap2;
          if constexpr (BG) {
            // the background's lap A and div A on the swamp layers
            if (live && k >= a.bg.ksw) {
              const long long ns = n2 * (L.nz - a.bg.ksw), qs = (long long)(k - a.bg.ksw) * n2 + (long long)j * L.nx + i;
              l0 = add(l0, __ldg(reinterpret_cast<const float2*>(a.bg.bL + qs)));
              l1 = add(l1, __ldg(reinterpret_cast<const float2*>(a.bg.bL + ns + qs)));
              l2 = add(l2, __ldg(reinterpret_cast<const float2*>(a.bg.bL + 2 * ns + qs)));
              divA = add(divA, __ldg(reinterpret_cast<const float2*>(a.bg.bL + 3 * ns + qs)));
            }
          }
          sw0 = mul(ews, l0);
          sw1 = mul(ews, l1);
          sw2 = fma2(mul(F2(ph.eta_s), wp), divA, mul(ews, l2));
        }
        if constexpr (BG) {
          B0 = add(B0, gB[0]);
          B1 = add(B1, gB[1]);
          B2 = add(B2, gB[2]);
          J0 = add(J0, gJ[0]);
          J1 = add(J1, gJ[1]);
          J2 = add(J2, gJ[2]);
        }
      }
      // u: dU[c][a] = d_a u_c, lap u, grad div u
      f2 U00, U10, U20, U21, lapU0, lapU1, lapU2, gdU0, gdU1, gdU2;
      {
        f2 xxUx, xxUy, xxUz, yyUz;
        dx_pair(Pk + UX * FP, a.cx, U00, &xxUx);
        dx_pair(Pk + UY * FP, a.cx, U10, &xxUy);
        dx_pair(Pk + UZ * FP, a.cx, U20, &xxUz);
        ds_pair(Pk + UZ * FP, BX, a.cy, U21, &yyUz);
        lapU0 = add(add(xxUx, yyUx), d2z[UX]);
        lapU1 = add(add(xxUy, yyUy), d2z[UY]);
        lapU2 = add(add(xxUz, yyUz), d2z[UZ]);
        gdU0 = add(add(xxUx, mxy[2]), mz[3]);
        gdU1 = add(add(mxy[3], yyUy), mz[4]);
        gdU2 = add(mz[5], d2z[UZ]);
      }
      const f2 U01 = dyUx, U02 = d1z[UX];
      const f2 U11 = dyUy, U12 = d1z[UY];
      const f2 U22 = d1z[UZ];
      // ln rho, ln T (perturbations about the background profiles)
      f2 gL0, gL1, lapL, gT0, gT1, lapT;
      {
        f2 xx, yy;
        dx_pair(Pk + LR * FP, a.cx, gL0, &xx);
        ds_pair(Pk + LR * FP, BX, a.cy, gL1, &yy);
        lapL = add(add(add(xx, yy), d2z[LR]), F2(d2lk));
        dx_pair(Pk + LT * FP, a.cx, gT0, &xx);
        ds_pair(Pk + LT * FP, BX, a.cy, gT1, &yy);
        lapT = add(add(add(xx, yy), d2z[LT]), F2(d2tk));
      }
      const f2 gL2 = add(d1z[LR], F2(dlk));
      const f2 gT2 = add(d1z[LT], F2(dtk));
      // RK accumulator of the pair (bounded wait; a time-out is recorded and
      // the step continues, so the CTA stays convergent)
      f2 dfo[NF];
      if (sub > 0) {
        const int sl = (k - k0) & 1;
        if (!zm::mbar_wait(&mbd[sl], (dphase >> sl) & 1u, a.wait_limit)) atomicOr(&a.ss->nonfinite, 2);
        dphase ^= 1u << sl;
        if (tid == 0) dpending &= ~(1u << sl);
        const float* dq = dfs + sl * DFT + ty * TX + 2 * tx;
#pragma unroll
        for (int f = 0; f < NF; ++f) dfo[f] = ld2(dq + f * TY * TX);
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) dfo[f] = F2(0.f);
      }

      if (live) {
        // ---- pointwise physics of the pair ----------------------------------
        const f2 A0 = vz[AX], A1 = vz[AY], A2 = vz[AZ];
        const f2 u0 = vz[UX], u1 = vz[UY], u2 = vz[UZ];
        const f2 Lr = add(F2(lbk), vz[LR]);
        const f2 Th = add(F2(tbk), vz[LT]);

        const f2 divU = add(add(U00, U11), U22);
        // exponentials and the reciprocal by the hardware approximations
        // (__expf: a few ulp plus about one ulp per unit of |x|; __fdividef:
        // 2 ulp), a few 1e-6 relative at the arguments of the stratified
        // box, against the 1e-4 of the FP32 path
        const f2 T = make_float2(__expf(Th.x), __expf(Th.y));
        const f2 rho1 = make_float2(__expf(-Lr.x), __expf(-Lr.y));
        const f2 eta = F2(ph.eta), nu = F2(ph.nu), gm1 = F2(ph.gm1);
        f2 out[NF];
        // induction
        out[AX] = add(dif(dif(mul(u1, B2), mul(u2, B1)), mul(eta, J0)), sw0);
        out[AY] = add(dif(dif(mul(u2, B0), mul(u0, B2)), mul(eta, J1)), sw1);
        out[AZ] = add(dif(dif(mul(u0, B1), mul(u1, B0)), mul(eta, J2)), sw2);
        // traceless rate of strain
        const f2 third = F2(1.f / 3.f), half = F2(0.5f), two = F2(2.f);
        const f2 s00 = dif(U00, mul(third, divU)), s11 = dif(U11, mul(third, divU)), s22 = dif(U22, mul(third, divU));
        const f2 s01 = mul(half, add(U01, U10));
        const f2 s02 = mul(half, add(U02, U20));
        const f2 s12 = mul(half, add(U12, U21));
        const f2 S2 = fma2(two, fma2(s01, s01, fma2(s02, s02, mul(s12, s12))),
                           fma2(s00, s00, fma2(s11, s11, mul(s22, s22))));
        const f2 SgL0 = fma2(s00, gL0, fma2(s01, gL1, mul(s02, gL2)));
        const f2 SgL1 = fma2(s01, gL0, fma2(s11, gL1, mul(s12, gL2)));
        const f2 SgL2 = fma2(s02, gL0, fma2(s12, gL1, mul(s22, gL2)));
        // Lorentz force
        const f2 F0 = dif(mul(J1, B2), mul(J2, B1));
        const f2 F1 = dif(mul(J2, B0), mul(J0, B2));
        const f2 Fz = dif(mul(J0, B1), mul(J1, B0));
        const f2 adv0 = fma2(u0, U00, fma2(u1, U01, mul(u2, U02)));
        const f2 adv1 = fma2(u0, U10, fma2(u1, U11, mul(u2, U12)));
        const f2 adv2 = fma2(u0, U20, fma2(u1, U21, mul(u2, U22)));
        out[UX] = add(dif(mul(F0, rho1), add(adv0, mul(T, add(gL0, gT0)))),
                      mul(nu, fma2(two, SgL0, fma2(third, gdU0, lapU0))));
        out[UY] = add(dif(mul(F1, rho1), add(adv1, mul(T, add(gL1, gT1)))),
                      mul(nu, fma2(two, SgL1, fma2(third, gdU1, lapU1))));
        out[UZ] = add(add(dif(mul(Fz, rho1), add(adv2, mul(T, add(gL2, gT2)))),
                          mul(nu, fma2(two, SgL2, fma2(third, gdU2, lapU2)))),
                      F2(ph.gz));
        // continuity
        const f2 ugL = fma2(u0, gL0, fma2(u1, gL1, mul(u2, gL2)));
        const f2 gLs = fma2(gL0, gL0, fma2(gL1, gL1, mul(gL2, gL2)));
        out[LR] = add(dif(mul(F2(ph.drho), add(lapL, gLs)), add(ugL, divU)), mul(mul(F2(ph.drho_s), w), lapL));
        // energy (ln T)
        const f2 ugT = fma2(u0, gT0, fma2(u1, gT1, mul(u2, gT2)));
        const f2 gTs = fma2(gT0, gT0, fma2(gT1, gT1, mul(gT2, gT2)));
        const f2 JJ = fma2(J0, J0, fma2(J1, J1, mul(J2, J2)));
        const f2 T1 = make_float2(__fdividef(1.f, T.x), __fdividef(1.f, T.y));
        const f2 heat = mul(mul(gm1, fma2(mul(eta, JJ), rho1, mul(two, mul(nu, S2)))), T1);
        const f2 ka = dif(mul(F2(2.5f), Th), Lr);
        const f2 kt = mul(F2(ph.gm1 * ph.kappa0), make_float2(__expf(ka.x), __expf(ka.y)));
        out[LT] = add(add(dif(heat, fma2(gm1, divU, ugT)), mul(kt, fma2(F2(3.5f), gTs, lapT))),
                      mul(mul(F2(ph.chi_s), w), lapT));
        if constexpr (NC) {
          if (k < ph.nc_k1)  // Newtonian cooling, one cell at a time
            out[LT] = add(out[LT], make_float2(nc_term<float>(ph, a.bg, L.nz, k, Lr.x, Th.x, nullptr, nullptr),
                                               nc_term<float>(ph, a.bg, L.nz, k, Lr.y, Th.y, nullptr, nullptr)));
        }

        // ---- nudging and boundary rows -----------------------------------------
        f2 tgx = F2(0.f), tgy = F2(0.f);
        if (ph.bcz == 0 && k == 0) {
          const long long q2 = (long long)j * L.nx + i;
          const f2 v0x = ld2(a.v0 + q2), v1x = ld2(a.v1 + q2);
          const f2 v0y = ld2(a.v0 + n2 + q2), v1y = ld2(a.v1 + n2 + q2);
          tgx = mul(F2(rr), fma2(F2(ss_), dif(v1x, v0x), v0x));
          tgy = mul(F2(rr), fma2(F2(ss_), dif(v1y, v0y), v0y));
          out[AX] = dif(out[AX], mul(F2(ph.tau_A), dif(A0, ld2(a.axt + q2))));
          out[AY] = dif(out[AY], mul(F2(ph.tau_A), dif(A1, ld2(a.ayt + q2))));
          out[UX] = dif(out[UX], mul(F2(ph.tau_u), dif(u0, tgx)));
          out[UY] = dif(out[UY], mul(F2(ph.tau_u), dif(u1, tgy)));
          out[UZ] = F2(0.f);
          out[LR] = F2(0.f);
        }
        if (ph.bcz == 0 && k == L.nz - 1) out[UZ] = F2(0.f);

        // ---- RK update and stores (pairs; periodic images) ---------------------
        // x images: pairs (0,1), (2,3) -> +nx; (nx-4, nx-3), (nx-2, nx-1) -> -nx
        // (the extra cell of each image pair lands in row padding)
        const int ox = i < NG ? L.nx : (i + 1 >= L.nx - NG ? -L.nx : 0);
        const long long oy = j < NG ? (long long)L.ny * L.mx : (j >= L.ny - NG ? -(long long)L.ny * L.mx : 0);
        const f2 vv[NF] = {A0, A1, A2, u0, u1, u2, vz[LR], vz[LT]};
        f2 vn[NF];
        {
          float* dq = a.df + cq;
          float* fq = a.fout + cq;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const f2 dfn = fma2(F2(alpha), dfo[f], mul(F2(dt), out[f]));
            if (sub < 2) *reinterpret_cast<f2*>(dq + f * L.fs) = dfn;
            vn[f] = fma2(F2(beta), dfn, vv[f]);
            if (!eval) *reinterpret_cast<f2*>(fq + f * L.fs) = vn[f];
          }
          if (!eval && (ox | (int)(oy != 0))) {
            // periodic images (pairs at the x, y edges only)
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              float* o = fq + f * L.fs;
              if (ox) *reinterpret_cast<f2*>(o + ox) = vn[f];
              if (oy) *reinterpret_cast<f2*>(o + oy) = vn[f];
              if (ox && oy) *reinterpret_cast<f2*>(o + ox + oy) = vn[f];
            }
          }
        }
        if (ph.bcz == 0 && k == 0) {
          // stateful u_x, u_y ghost rows below the photosphere: nudging only;
          // their values are the TMEM copies of planes -1 .. -3
#pragma unroll
          for (int m = 1; m <= NG; ++m) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const long long q = L.at(UX + cc, -m, j, i);
              const f2 u = cc == 0 ? gux[m - 1] : guy[m - 1];
              const f2 rh = mul(F2(-ph.tau_u), dif(u, cc == 0 ? tgx : tgy));
              const f2 dfn = fma2(F2(alpha), sub > 0 ? ld2(a.df + q) : F2(0.f), mul(F2(dt), rh));
              if (sub < 2) *reinterpret_cast<f2*>(a.df + q) = dfn;
              if (!eval) {
                const f2 vn = fma2(F2(beta), dfn, u);
                *reinterpret_cast<f2*>(a.fout + q) = vn;
                if (ox) *reinterpret_cast<f2*>(a.fout + q + ox) = vn;
                if (oy) *reinterpret_cast<f2*>(a.fout + q + oy) = vn;
                if (ox && oy) *reinterpret_cast<f2*>(a.fout + q + ox + oy) = vn;
              }
            }
          }
        }
      }
    }
    if (!bad) {
      // all threads are past the last centre: the next item may refill any slot
      if (a.dyn && tid == 0) s_next = next;
      __syncthreads();
      item = a.dyn ? s_next : item + (int)gridDim.x;
    }
  }
  if (bad && tid == 0) {
    // a ring wait timed out: record it and drain the copies in flight (bounded)
    atomicOr(&a.ss->nonfinite, 2);
    for (int s = 0; s < NR; ++s)
      if (pending & (1u << s)) zm::mbar_wait(&mbar[s], (phase >> s) & 1u, a.wait_limit);
    for (int s = 0; s < 2; ++s)
      if (dpending & (1u << s)) zm::mbar_wait(&mbd[s], (dphase >> s) & 1u, a.wait_limit);
  }
  tm_wait_st();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

}  // namespace pair

bool rk_pair_supported(const Layout& L) { return L.nx % 2 == 0 && L.nx >= 8 && L.ny >= 6; }

// persistent CTAs of the pair kernels on the current device (two per SM: the
// shared ring admits no third, and TMEM holds two), after setting their
// shared-memory limit there
static int pair_ctas() {
  static PerDevice<int> ctas;
  return ctas.get([] {
    auto attr = [](const void* fn) {
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair::SMEM_BYTES);
    };
    attr((const void*)pair::rk_pair_kernel<false, false, false, false>);
    attr((const void*)pair::rk_pair_kernel<false, true, false, false>);
    attr((const void*)pair::rk_pair_kernel<false, false, true, false>);
    attr((const void*)pair::rk_pair_kernel<false, true, true, false>);
    attr((const void*)pair::rk_pair_kernel<false, false, false, true>);
    attr((const void*)pair::rk_pair_kernel<false, true, false, true>);
    attr((const void*)pair::rk_pair_kernel<false, false, true, true>);
    attr((const void*)pair::rk_pair_kernel<false, true, true, true>);
    attr((const void*)pair::rk_pair_kernel<true, false, false, false>);
    return 2 * sm_count();
  });
}

static pair::Args pair_args(const Layout& L, const Phys<float>& ph, const Background<float>& bg, const float* wtab,
                            const float* wptab, StepState* ss, int sub, double dx, double dy, double dz) {
  const int ctas = pair_ctas();
  pair::Args a{};
  a.wait_limit = zm::WAIT_LIMIT;
  a.skip_plane = INT_MIN;
  a.L = L;
  a.ph = ph;
  a.bg = bg;
  a.wtab = wtab;
  a.wptab = wptab;
  a.ss = ss;
  a.sub = sub;
  a.ntx = (L.nx + pair::TX - 1) / pair::TX;
  a.nty = (L.ny + pair::TY - 1) / pair::TY;
  const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
  const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0, 2.0 / 180.0};
  auto coef = [&](double h) {
    pair::Coef c;
    c.c1 = make_float2((float)(W1[1] / h), (float)(W1[1] / h));
    c.c2 = make_float2((float)(W1[2] / h), (float)(W1[2] / h));
    c.c3 = make_float2((float)(W1[3] / h), (float)(W1[3] / h));
    c.e0 = make_float2((float)(W2[0] / (h * h)), (float)(W2[0] / (h * h)));
    c.e1 = make_float2((float)(W2[1] / (h * h)), (float)(W2[1] / (h * h)));
    c.e2 = make_float2((float)(W2[2] / (h * h)), (float)(W2[2] / (h * h)));
    c.e3 = make_float2((float)(W2[3] / (h * h)), (float)(W2[3] / (h * h)));
    return c;
  };
  a.cx = coef(dx);
  a.cy = coef(dy);
  a.cz = coef(dz);
  const int tiles = a.ntx * a.nty;
  a.kchunk = zm::zchunk(L.nz, tiles, ctas);
  a.nch = (L.nz + a.kchunk - 1) / a.kchunk;
  return a;
}

void launch_rk_pair(const CUtensorMap* tm, const CUtensorMap* tmd, const Layout& L, const Phys<float>& ph,
                    const Background<float>& bg, float* fout, float* df, const float* wtab, const float* wptab,
                    const Driver& drv, StepState* ss, int sub, double dx, double dy, double dz, cudaStream_t st,
                    int skip_plane, int wait_limit) {
  pair::Args a = pair_args(L, ph, bg, wtab, wptab, ss, sub, dx, dy, dz);
  if (skip_plane != INT_MIN) {
    a.skip_plane = skip_plane;
    a.wait_limit = wait_limit;
  }
  a.fout = fout;
  a.df = df;
  a.axt = (const float*)drv.axt;
  a.ayt = (const float*)drv.ayt;
  a.v0 = (const float*)drv.v0;
  a.v1 = (const float*)drv.v1;
  const int nitems = a.ntx * a.nty * a.nch;
  const int grid = nitems < pair_ctas() ? nitems : pair_ctas();
  // claimed work items where a CTA has a dozen or more: there the grid
  // stride's imbalance outweighs the claims (1024 x 1024 x 256: step 4 %
  // faster; at 256^3, six items per CTA, the stride is 2 % faster)
  a.dyn = nitems >= 12 * grid;
  // the instantiation for the options in use (cooling, A about a
  // background, non-uniform vertical grid)
  const int opt = (ph.nc_k1 > 0 ? 1 : 0) | (bg.bB != nullptr ? 2 : 0) | (bg.zm1 != nullptr ? 4 : 0);
  const dim3 g(grid), b(pair::NT);
  if (a.dyn) cudaMemsetAsync(&ss->items, 0, sizeof(int), st);
  switch (opt) {
    case 0: pair::rk_pair_kernel<false, false, false, false><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 1: pair::rk_pair_kernel<false, true, false, false><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 2: pair::rk_pair_kernel<false, false, true, false><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 3: pair::rk_pair_kernel<false, true, true, false><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 4: pair::rk_pair_kernel<false, false, false, true><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 5: pair::rk_pair_kernel<false, true, false, true><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    case 6: pair::rk_pair_kernel<false, false, true, true><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
    default: pair::rk_pair_kernel<false, true, true, true><<<g, b, pair::SMEM_BYTES, st>>>(*tm, *tmd, a); break;
  }
}

void launch_adj_point_pair(const CUtensorMap* tm, const CUtensorMap* tmd, const Layout& L, const Phys<float>& ph,
                           const Background<float>& bg, const float* dbar, float* coef, double* thbar,
                           const float* wtab, const float* wptab, StepState* ss, int sub, double dx, double dy,
                           double dz, cudaStream_t st) {
  pair::Args a = pair_args(L, ph, bg, wtab, wptab, ss, sub, dx, dy, dz);
  a.dbar = dbar;
  a.coef = coef;
  a.thbar = thbar;
  const int nitems = a.ntx * a.nty * a.nch;
  const int grid = nitems < pair_ctas() ? nitems : pair_ctas();
  a.dyn = nitems >= 12 * grid;
  if (a.dyn) cudaMemsetAsync(&ss->items, 0, sizeof(int), st);
  pair::rk_pair_kernel<true, false, false, false><<<grid, pair::NT, pair::SMEM_BYTES, st>>>(*tm, *tmd, a);
}

}  // namespace mhd
