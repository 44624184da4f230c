// mhd_abg.cu -- the vector potential stored as a perturbation about a fixed
// background field (params a_background).
//
// Where |A| is large (hundreds in the production-size box, whose sigma = 40
// cell pair spans 160 length units at dx = 4), FP32 storage of A rounds it by
// 2^-24 |A|, and the second differences of J = grad div A - lap A turn that
// rounding into a spurious current that the Lorentz force accelerates in the
// low-density corona.  As with ln rho and ln T (stored about their initial
// profiles), the state then holds A' = A - A_bg and the kernels add the
// background's contribution to every term that is linear in A: B and J per
// cell, and lap A, div A on the swamp layers (Eq. 18).  The discrete equations
// are unchanged; FP32 rounding scales with |A'|.
//
// Set-up (once per mhd_set_a_background): the FP64 background is unpacked into
// a padded FP64 scratch (fields 0..2 of the state layout, in the RK
// accumulator's memory), its ghosts are filled by the state's own boundary
// rules in FP64 (potential-field extrapolations, or periodic copies), and the
// tables below are formed with FP64 sixth-order stencils and stored in the
// state precision.
#include "mhd_internal.h"

namespace mhd {

// interior cell (k, j, i) and its periodic x,y images inside the padded plane
template <typename R>
__device__ __forceinline__ void put_images(const Layout& L, R* __restrict__ f, int fl, int k, int j, int i, R v) {
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

// packed [3][nz][ny][nx] -> fields 0..2 of the padded layout (interior and
// x,y images); used for the FP64 background and for the perturbation A'
template <typename Rin, typename R>
__global__ void abg_unpack_kernel(Layout L, const Rin* __restrict__ in, R* __restrict__ a) {
  const long long n3 = (long long)L.nx * L.ny * L.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * n3;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % L.nx);
    long long r = q / L.nx;
    const int j = (int)(r % L.ny);
    r /= L.ny;
    const int k = (int)(r % L.nz);
    const int fl = (int)(r / L.nz);
    put_images<R>(L, a, fl, k, j, i, (R)in[q]);
  }
}

// periodic copies in z of fields 0..2 (bc_z = 1), over whole padded planes
__global__ void abg_zper_kernel(Layout L, double* __restrict__ a) {
  const int pw = L.nx + 2 * NG, ph = L.ny + 2 * NG;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= pw * ph) return;
  const int i = q % pw - NG, j = q / pw - NG, nz = L.nz;
  for (int fl = 0; fl < 3; ++fl)
    for (int m = 1; m <= NG; ++m) {
      a[L.at(fl, -m, j, i)] = a[L.at(fl, nz - m, j, i)];
      a[L.at(fl, nz - 1 + m, j, i)] = a[L.at(fl, m - 1, j, i)];
    }
}

// Tables of the ghost-filled FP64 background at interior cells: B = curl A,
// J = grad div A - lap A, and on layers k >= ksw lap A and div A; the
// photospheric A_x, A_y in FP64 (for the nudging target difference).  zm: on
// a non-uniform vertical grid the FP64 metric per interior layer ([2][nz]:
// dxi/dz, then r21 with D_z^2 f = (dxi/dz)^2 D_xi^2 f + r21 D_z f); null on
// the uniform grid.
template <typename R>
__global__ void __launch_bounds__(256) abg_tables_kernel(Layout L, double idx, double idy, double idz,
                                                         const double* __restrict__ zm,
                                                         const double* __restrict__ a, R* __restrict__ bB,
                                                         R* __restrict__ bJ, R* __restrict__ bL, int ksw,
                                                         double* __restrict__ a0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  const long long st[3] = {1, L.sy(), L.sz()};
  const double m1 = zm ? zm[k] : idz, r21 = zm ? zm[L.nz + k] : 0.0;
  const double inv[3] = {idx, idy, m1};
  const double inv2[3] = {idx * idx, idy * idy, m1 * m1};
  const double* p[3];
  for (int c = 0; c < 3; ++c) p[c] = a + L.at(c, k, j, i);
  double d[3][3];  // d[c][x] = d_x A_c
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) d[c][x] = d1<double>(p[c], st[x], inv[x]);
  // second derivatives, with the vertical metric's first-derivative term
  auto dd = [&](int c, int x) { return d2<double>(p[c], st[x], inv2[x]) + (x == 2 ? r21 * d[c][2] : 0.0); };
  double lap[3], gd[3];
  for (int c = 0; c < 3; ++c) {
    lap[c] = 0.0;
    for (int x = 0; x < 3; ++x) lap[c] += dd(c, x);
  }
  for (int x = 0; x < 3; ++x) {
    gd[x] = 0.0;
    for (int c = 0; c < 3; ++c) gd[x] += c == x ? dd(c, x) : d11<double>(p[c], st[x], st[c], inv[x], inv[c]);
  }
  const long long n2 = (long long)L.nx * L.ny, n3 = n2 * L.nz;
  const long long q = (long long)k * n2 + (long long)j * L.nx + i;
  bB[q] = (R)(d[2][1] - d[1][2]);
  bB[n3 + q] = (R)(d[0][2] - d[2][0]);
  bB[2 * n3 + q] = (R)(d[1][0] - d[0][1]);
  for (int c = 0; c < 3; ++c) bJ[c * n3 + q] = (R)(gd[c] - lap[c]);
  if (k >= ksw) {
    const long long ns = n2 * (L.nz - ksw), qs = (long long)(k - ksw) * n2 + (long long)j * L.nx + i;
    for (int c = 0; c < 3; ++c) bL[c * ns + qs] = (R)lap[c];
    bL[3 * ns + qs] = (R)(d[0][0] + d[1][1] + d[2][2]);
  }
  if (k == 0) {
    a0[(long long)j * L.nx + i] = *p[0];
    a0[n2 + (long long)j * L.nx + i] = *p[1];
  }
}

// the padded FP64 background (fields 0..2, ghosts and rims included) rounded
// to the state precision
template <typename R>
__global__ void abg_round_kernel(const double* __restrict__ a, R* __restrict__ out, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (R)a[q];
}

// nudging target relative to the background at the photosphere, formed in
// FP64: rel = A_target - A_bg(k = 0), both components
template <typename R>
__global__ void abg_target_kernel(const double* __restrict__ at, const double* __restrict__ a0, R* __restrict__ rel,
                                  long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    rel[q] = (R)(at[q] - a0[q]);
}

template <typename R>
__global__ void widen_kernel(const R* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (double)in[q];
}

void launch_abg_unpack64(const Layout& L, const double* in, double* a, cudaStream_t st) {
  abg_unpack_kernel<double, double><<<1216, 256, 0, st>>>(L, in, a);
}

template <typename R>
void launch_abg_pert(const Layout& L, const R* in, R* f, cudaStream_t st) {
  abg_unpack_kernel<R, R><<<1216, 256, 0, st>>>(L, in, f);
}

void launch_abg_zper(const Layout& L, double* a, cudaStream_t st) {
  const int n = (L.nx + 2 * NG) * (L.ny + 2 * NG);
  abg_zper_kernel<<<(n + 255) / 256, 256, 0, st>>>(L, a);
}

template <typename R>
void launch_abg_tables(const Layout& L, double dx, double dy, double dz, const double* zm, const double* a, R* bB,
                       R* bJ, R* bL, int ksw, double* a0, R* abg, cudaStream_t st) {
  dim3 blk(32, 8, 1), grd((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
  abg_tables_kernel<R><<<grd, blk, 0, st>>>(L, 1.0 / dx, 1.0 / dy, 1.0 / dz, zm, a, bB, bJ, bL, ksw, a0);
  abg_round_kernel<R><<<1216, 256, 0, st>>>(a, abg, 3 * L.fs);
}

template <typename R>
void launch_abg_target(const double* at, const double* a0, R* rel, long long n, cudaStream_t st) {
  abg_target_kernel<R><<<(int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216), 256, 0, st>>>(at, a0, rel, n);
}

template <typename R>
void launch_widen(const R* in, double* out, long long n, cudaStream_t st) {
  widen_kernel<R><<<(int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216), 256, 0, st>>>(in, out, n);
}

#define INST(R)                                                                                               \
  template void launch_abg_pert<R>(const Layout&, const R*, R*, cudaStream_t);                               \
  template void launch_abg_tables<R>(const Layout&, double, double, double, const double*, const double*, R*,  \
                                     R*, R*, int,                                                             \
                                     double*, R*, cudaStream_t);                                             \
  template void launch_abg_target<R>(const double*, const double*, R*, long long, cudaStream_t);             \
  template void launch_widen<R>(const R*, double*, long long, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mhd
