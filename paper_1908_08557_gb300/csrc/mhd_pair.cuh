// mhd_pair.cuh -- packed FP32 pairs (f32x2: FFMA2, FADD2, FMUL2) and the
// sixth-order stencils of two x-adjacent cells, shared by the z-march kernels
// that work on cell pairs (the right-hand side / RK kernel, its adjoint point
// mode, the adjoint gather).
#pragma once
#include <cuda_runtime.h>

namespace mhd {
namespace pk {

typedef float2 f2;
__host__ __device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b, one rounding
__device__ __forceinline__ f2 dif(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.f), a); }
__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }

// stencil weights divided by the spacing (D1) or its square (D2), as pairs
struct Coef {
  f2 c1, c2, c3;        // D1 weights / spacing
  f2 e0, e1, e2, e3;    // D2 weights / spacing^2
};

// ---- stencils on a box row / column at an even x position -----------------
// first and second x derivatives of the cell pair at p (p even, p - 4 .. p + 5 in the row)
__device__ __forceinline__ void dx_pair(const float* p, const Coef& c, f2& d1, f2* d2) {
  const f2 m4 = ld2(p - 4), m2 = ld2(p - 2), z0 = ld2(p), p2 = ld2(p + 2), p4 = ld2(p + 4);
  const f2 om3 = make_float2(m4.y, m2.x), om1 = make_float2(m2.y, z0.x);
  const f2 op1 = make_float2(z0.y, p2.x), op3 = make_float2(p2.y, p4.x);
  d1 = fma2(c.c1, dif(op1, om1), fma2(c.c2, dif(p2, m2), mul(c.c3, dif(op3, om3))));
  if (d2) *d2 = fma2(c.e0, z0, fma2(c.e1, add(op1, om1), fma2(c.e2, add(p2, m2), mul(c.e3, add(op3, om3)))));
}
// first and second derivatives along a stride s (in floats) of the pair at p
__device__ __forceinline__ void ds_pair(const float* p, int s, const Coef& c, f2& d1, f2* d2) {
  const f2 z0 = ld2(p), a1 = ld2(p + s), b1 = ld2(p - s), a2 = ld2(p + 2 * s), b2 = ld2(p - 2 * s),
           a3 = ld2(p + 3 * s), b3 = ld2(p - 3 * s);
  d1 = fma2(c.c1, dif(a1, b1), fma2(c.c2, dif(a2, b2), mul(c.c3, dif(a3, b3))));
  if (d2) *d2 = fma2(c.e0, z0, fma2(c.e1, add(a1, b1), fma2(c.e2, add(a2, b2), mul(c.e3, add(a3, b3)))));
}

}  // namespace pk
}  // namespace mhd
