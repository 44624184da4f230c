// mhd_gran.cu -- the granulation driver (Sect. 2.3, Eqs. 1-4) on the GPU.
//
// State: one slot per pixel (occupancy, t0, T, v_max, t_max), so granules
// need no list, compaction or host bookkeeping.
//
// Update (the population at time t):
//   1. expire:  occ = 0 where t - t0 - t_max > t_max (Eq. 2 is back at v_min)
//   2. seed:    a pixel within r_inner of a live centre is out, the rest
//               undecided
//   3. rounds:  join: an undecided pixel with no undecided pixel of smaller
//               (key, index) within r_inner, and no member there, becomes a
//               member; exclude: an undecided pixel with a member within
//               r_inner is out.  Repeated until nothing is undecided, this
//               gives exactly the set the sequential visit in (key, index)
//               order accepts (the first undecided pixel in that order joins
//               every round, so the rounds end).
//   4. birth:   members become granules with the draws at their pixel.
// Velocity at time t:
//   5. amp:     per pixel, Eq. 2 of its granule (0 where none)
//   6. render:  v_gran(p) = sum over lane offsets o of amp(p - o) w(o), with
//               w(o) = profile(|o|) o / |o| tabulated on the host
//   7. FFT:     the filtered rotational part (Eq. 3), packed plane v_x + i v_y
//   8. combine: v_vor = v_gran + f_rot v_rot', with block sums of |v|^2 of
//               both fields; one block totals them in a fixed order; scale
//               v_vor to the rms of v_gran (Eq. 4) into the caller's array.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mhd.h"
#include "mhd_internal.h"

namespace mhd {
namespace {

constexpr int GT = 256;             // threads per block of the pixel kernels
constexpr int GMAX_PX = 64;         // largest disk radius in pixels
constexpr int UNDECIDED = 0, MEMBER = 1, OUT = 2;

struct GranDev {
  int nx, ny;
  int* occ;
  double *t0, *life, *vmax, *tmax;  // [ny][nx] each
  int* mis;
  double* amp;
  double* vg;  // [2][ny][nx]
  double* vr;  // [2][ny][nx]: the rotational part, then v_vor
  const int2* off_in;
  int n_in;
  const int2* off_l;
  const double2* w_l;
  int n_l;
  double* part;  // [2][nblk] block sums
  double* tot;   // [2]: scale, spare
  int* cnt;
};

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__global__ void __launch_bounds__(GT) expire_kernel(GranDev g, double t) {
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= g.nx * g.ny) return;
  if (g.occ[p] && t - g.t0[p] - g.tmax[p] > g.tmax[p]) {
    g.occ[p] = 0;
    g.t0[p] = g.life[p] = g.vmax[p] = g.tmax[p] = 0.0;
  }
}

__global__ void __launch_bounds__(GT) seed_kernel(GranDev g) {
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= g.nx * g.ny) return;
  const int y = p / g.nx, x = p - y * g.nx;
  bool blocked = g.occ[p] != 0;
  for (int n = 0; n < g.n_in && !blocked; ++n) {
    const int2 o = __ldg(g.off_in + n);
    blocked = g.occ[wrap(y + o.y, g.ny) * g.nx + wrap(x + o.x, g.nx)] != 0;
  }
  g.mis[p] = blocked ? OUT : UNDECIDED;
}

// Reads of neighbours race with their writes in the same launch; either
// value gives the same decision (a neighbour that joins now precedes p, so
// p does not join whether it reads UNDECIDED or MEMBER).
__global__ void __launch_bounds__(GT) join_kernel(GranDev g, const unsigned* __restrict__ keys) {
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= g.nx * g.ny) return;
  if (g.mis[p] != UNDECIDED) return;
  const int y = p / g.nx, x = p - y * g.nx;
  const unsigned kp = keys[p];
  for (int n = 0; n < g.n_in; ++n) {
    const int2 o = __ldg(g.off_in + n);
    const int q = wrap(y + o.y, g.ny) * g.nx + wrap(x + o.x, g.nx);
    const int s = ((volatile int*)g.mis)[q];
    if (s == MEMBER) return;
    if (s == UNDECIDED) {
      const unsigned kq = keys[q];
      if (kq < kp || (kq == kp && q < p)) return;
    }
  }
  g.mis[p] = MEMBER;
}

__global__ void __launch_bounds__(GT) exclude_kernel(GranDev g) {
  const int p = blockIdx.x * GT + threadIdx.x;
  int undecided = 0;
  if (p < g.nx * g.ny && g.mis[p] == UNDECIDED) {
    const int y = p / g.nx, x = p - y * g.nx;
    bool hit = false;
    for (int n = 0; n < g.n_in && !hit; ++n) {
      const int2 o = __ldg(g.off_in + n);
      hit = g.mis[wrap(y + o.y, g.ny) * g.nx + wrap(x + o.x, g.nx)] == MEMBER;
    }
    if (hit) g.mis[p] = OUT;
    else undecided = 1;
  }
  const int c = __syncthreads_count(undecided);
  if (threadIdx.x == 0 && c) atomicAdd(g.cnt, c);
}

__global__ void __launch_bounds__(GT) birth_kernel(GranDev g, mhd_gran_params gp, double t,
                                                   const double* __restrict__ c_life,
                                                   const double* __restrict__ c_amp) {
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= g.nx * g.ny || g.mis[p] != MEMBER) return;
  const double cl = fmin(1.0, fmax(-1.0, c_life[p]));
  const double ca = fmin(1.0, fmax(-1.0, c_amp[p]));
  const double T = gp.lifetime * (1.0 + gp.lifetime_spread * cl);
  const double vm = gp.v0 * (1.0 + gp.amp_spread * ca);
  g.occ[p] = 1;
  g.t0[p] = t;
  g.life[p] = T;
  g.vmax[p] = vm;
  g.tmax[p] = T * sqrt(fabs(log(gp.vmin_frac * gp.v0 / vm)));  // Eq. 1
}

__global__ void __launch_bounds__(GT) amp_kernel(GranDev g, double t) {
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= g.nx * g.ny) return;
  double a = 0.0;
  if (g.occ[p]) {
    const double s = (t - g.t0[p] - g.tmax[p]) / g.life[p];
    a = g.vmax[p] * exp(-s * s);  // Eq. 2
  }
  g.amp[p] = a;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < GT / 32; ++i) s += sh[i];
  return s;
}

// v_gran at pixel p: the granule centred at p - o contributes amp w(o).
// Block sums of |v_gran|^2 into part[0][block].
__global__ void __launch_bounds__(GT) render_kernel(GranDev g) {
  __shared__ double sh[GT / 32];
  const int N = g.nx * g.ny;
  const int p = blockIdx.x * GT + threadIdx.x;
  double e = 0.0;
  if (p < N) {
    const int y = p / g.nx, x = p - y * g.nx;
    double vx = 0.0, vy = 0.0;
    for (int n = 0; n < g.n_l; ++n) {
      const int2 o = __ldg(g.off_l + n);
      const double a = __ldg(g.amp + wrap(y - o.y, g.ny) * g.nx + wrap(x - o.x, g.nx));
      if (a != 0.0) {
        const double2 w = __ldg(g.w_l + n);
        vx = fma(a, w.x, vx);
        vy = fma(a, w.y, vy);
      }
    }
    g.vg[p] = vx;
    g.vg[N + p] = vy;
    e = vx * vx + vy * vy;
  }
  const double s = block_sum(e, sh);
  if (threadIdx.x == 0) g.part[blockIdx.x] = s;
}

// v_vor = v_gran + f_rot v_rot' into vr; block sums of |v_vor|^2 into part[1][block]
__global__ void __launch_bounds__(GT) combine_kernel(GranDev g, double f_rot, int nblk) {
  __shared__ double sh[GT / 32];
  const int N = g.nx * g.ny;
  const int p = blockIdx.x * GT + threadIdx.x;
  double e = 0.0;
  if (p < N) {
    const double wx = g.vg[p] + f_rot * g.vr[p];
    const double wy = g.vg[N + p] + f_rot * g.vr[N + p];
    g.vr[p] = wx;
    g.vr[N + p] = wy;
    e = wx * wx + wy * wy;
  }
  const double s = block_sum(e, sh);
  if (threadIdx.x == 0) g.part[nblk + blockIdx.x] = s;
}

// one block: totals of both block-sum rows in a fixed order, the Eq. 4 scale
__global__ void __launch_bounds__(GT) total_kernel(GranDev g, int nblk) {
  __shared__ double sh[GT / 32];
  double sv = 0.0, sw = 0.0;
  for (int i = threadIdx.x; i < nblk; i += GT) {
    sv += g.part[i];
    sw += g.part[nblk + i];
  }
  const double tv = block_sum(sv, sh);
  __syncthreads();
  const double tw = block_sum(sw, sh);
  if (threadIdx.x == 0) g.tot[0] = tw > 0.0 ? sqrt(tv / tw) : 0.0;
}

template <typename R>
__global__ void __launch_bounds__(GT) scale_kernel(GranDev g, R* __restrict__ v) {
  const int N = g.nx * g.ny;
  const int p = blockIdx.x * GT + threadIdx.x;
  if (p >= N) return;
  const double s = g.tot[0];
  v[p] = (R)(g.vr[p] * s);
  v[N + p] = (R)(g.vr[N + p] * s);
}

// ---- host side ---------------------------------------------------------------

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int lg2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// disk offsets (o != 0) with |o| < r, |o| = sqrt((o_x dx)^2 + (o_y dy)^2)
std::vector<int2> disk(double r, double dx, double dy) {
  std::vector<int2> out;
  const int mx = (int)std::ceil(r / dx), my = (int)std::ceil(r / dy);
  for (int oy = -my; oy <= my; ++oy)
    for (int ox = -mx; ox <= mx; ++ox) {
      if (ox == 0 && oy == 0) continue;
      const double ex = ox * dx, ey = oy * dy;
      if (ex * ex + ey * ey < r * r) out.push_back(make_int2(ox, oy));
    }
  return out;
}

const char* check(int nx, int ny, double dx, double dy, const mhd_gran_params* gp) {
  if (!gp) return "gran params are NULL";
  if (!pow2(nx) || !pow2(ny) || nx < 8 || ny < 8 || nx > 1024 || ny > 1024)
    return "nx, ny must be powers of two in [8, 1024]";
  if (!(dx > 0.0) || !(dy > 0.0)) return "dx, dy must be positive";
  if (!(gp->r_inner > 0.0) || !(gp->r_granule > 0.0) || !(gp->r_lane > gp->r_granule))
    return "need 0 < r_inner and 0 < r_granule < r_lane";
  const double rmax = gp->r_inner > gp->r_lane ? gp->r_inner : gp->r_lane;
  if (!(rmax < 0.5 * nx * dx) || !(rmax < 0.5 * ny * dy)) return "r_inner and r_lane must be below half the plane";
  if (rmax / dx > GMAX_PX || rmax / dy > GMAX_PX) return "r_inner and r_lane must span at most 64 pixels";
  if (!(gp->v0 > 0.0) || !(gp->lifetime > 0.0)) return "v0 and lifetime must be positive";
  if (!(gp->lifetime_spread >= 0.0 && gp->lifetime_spread < 1.0) ||
      !(gp->amp_spread >= 0.0 && gp->amp_spread < 1.0))
    return "spreads must lie in [0, 1)";
  if (!(gp->vmin_frac > 0.0 && gp->vmin_frac < 1.0 - gp->amp_spread))
    return "vmin_frac must lie in (0, 1 - amp_spread)";
  if (!std::isfinite(gp->f_rot)) return "f_rot must be finite";
  return nullptr;
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

struct Layout2 {
  size_t occ, par, mis, amp, vg, vr, keys, cl, ca, twx, twy, ktx, kty, P, Q, off_in, off_l, w_l, part, tot, cnt;
  size_t total;
  int n_in, n_l, nblk;
};

Layout2 carve(int nx, int ny, double dx, double dy, const mhd_gran_params* gp) {
  Layout2 o;
  const size_t N = (size_t)nx * ny;
  o.n_in = (int)disk(gp->r_inner, dx, dy).size();
  o.n_l = (int)disk(gp->r_lane, dx, dy).size();
  o.nblk = (int)((N + GT - 1) / GT);
  Carve c;
  o.occ = c.take(N * 4);
  o.par = c.take(4 * N * 8);
  o.mis = c.take(N * 4);
  o.amp = c.take(N * 8);
  o.vg = c.take(2 * N * 8);
  o.vr = c.take(2 * N * 8);
  o.keys = c.take(N * 4);
  o.cl = c.take(N * 8);
  o.ca = c.take(N * 8);
  o.twx = c.take((size_t)nx * 16);
  o.twy = c.take((size_t)ny * 16);
  o.ktx = c.take((size_t)nx * 8);
  o.kty = c.take((size_t)ny * 8);
  o.P = c.take(N * 16);
  o.Q = c.take(N * 16);
  o.off_in = c.take((size_t)(o.n_in > 0 ? o.n_in : 1) * 8);
  o.off_l = c.take((size_t)o.n_l * 8);
  o.w_l = c.take((size_t)o.n_l * 16);
  o.part = c.take((size_t)2 * o.nblk * 8);
  o.tot = c.take(2 * 8);
  o.cnt = c.take(8);
  o.total = c.off;
  return o;
}

}  // namespace
}  // namespace mhd

using namespace mhd;

struct mhd_gran_ctx {
  int nx, ny;
  double dx, dy;
  mhd_gran_params gp;
  char* ws;
  Layout2 o;
  GranDev g;
  FFTPlan fp;
  cudaStream_t st;
  long long launches = 0;
  char err[512] = "no error";
};

static int gfail(mhd_gran_ctx* g, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (g) snprintf(g->err, sizeof g->err, "%s", buf);
  else set_global_error("%s", buf);
  return code;
}

static int gcheck(mhd_gran_ctx* g, cudaError_t e, const char* what) {
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(g, MHD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return MHD_OK;
}

extern "C" size_t mhd_gran_workspace_bytes(int nx, int ny, double dx, double dy, const mhd_gran_params* gp) {
  if (check(nx, ny, dx, dy, gp)) return 0;
  return carve(nx, ny, dx, dy, gp).total;
}

extern "C" int mhd_gran_create(int nx, int ny, double dx, double dy, const mhd_gran_params* gp, void* workspace,
                               size_t ws_bytes, void* stream, mhd_gran_handle* out) {
  if (!out) return gfail(nullptr, MHD_ERR_ARG, "out is NULL");
  *out = nullptr;
  const char* bad = check(nx, ny, dx, dy, gp);
  if (bad) return gfail(nullptr, MHD_ERR_ARG, "%s", bad);
  const Layout2 o = carve(nx, ny, dx, dy, gp);
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < o.total)
    return gfail(nullptr, MHD_ERR_WORKSPACE, "workspace must be 256-byte aligned with at least %zu bytes", o.total);
  mhd_gran_ctx* g = new mhd_gran_ctx;
  g->nx = nx;
  g->ny = ny;
  g->dx = dx;
  g->dy = dy;
  g->gp = *gp;
  g->ws = (char*)workspace;
  g->o = o;
  g->st = (cudaStream_t)stream;
  const size_t N = (size_t)nx * ny;
  GranDev& d = g->g;
  d.nx = nx;
  d.ny = ny;
  d.occ = (int*)(g->ws + o.occ);
  d.t0 = (double*)(g->ws + o.par);
  d.life = d.t0 + N;
  d.vmax = d.t0 + 2 * N;
  d.tmax = d.t0 + 3 * N;
  d.mis = (int*)(g->ws + o.mis);
  d.amp = (double*)(g->ws + o.amp);
  d.vg = (double*)(g->ws + o.vg);
  d.vr = (double*)(g->ws + o.vr);
  d.off_in = (const int2*)(g->ws + o.off_in);
  d.n_in = o.n_in;
  d.off_l = (const int2*)(g->ws + o.off_l);
  d.w_l = (const double2*)(g->ws + o.w_l);
  d.n_l = o.n_l;
  d.part = (double*)(g->ws + o.part);
  d.tot = (double*)(g->ws + o.tot);
  d.cnt = (int*)(g->ws + o.cnt);
  FFTPlan& fp = g->fp;
  memset(&fp, 0, sizeof fp);
  fp.nx = nx;
  fp.ny = ny;
  fp.lognx = lg2(nx);
  fp.logny = lg2(ny);
  fp.twx = (const double2*)(g->ws + o.twx);
  fp.twy = (const double2*)(g->ws + o.twy);
  fp.ktx = (const double*)(g->ws + o.ktx);
  fp.kty = (const double*)(g->ws + o.kty);
  fp.P = (double2*)(g->ws + o.P);
  fp.Q = (double2*)(g->ws + o.Q);
  fp.p0 = 0;
  fp.knx = M_PI / dx;
  fp.kny = M_PI / dy;
  // host tables: twiddles, signed wavenumbers 2 pi m / L, disk offsets and
  // the lane weights profile(|o|) o / |o| (linear rise to r_granule, cos^2
  // fall to r_lane)
  int rc = MHD_OK;
  for (int axis = 0; axis < 2 && rc == MHD_OK; ++axis) {
    const int n = axis == 0 ? nx : ny;
    const double L = n * (axis == 0 ? dx : dy);
    std::vector<double> tw((size_t)2 * n), k((size_t)n);
    for (int r = 0; r < n; ++r) {
      tw[2 * r] = cos(2.0 * M_PI * r / n);
      tw[2 * r + 1] = -sin(2.0 * M_PI * r / n);
      k[r] = 2.0 * M_PI * (2 * r > n ? r - n : r) / L;
    }
    rc = gcheck(g, cudaMemcpy((void*)(axis == 0 ? fp.twx : fp.twy), tw.data(), (size_t)n * 16,
                              cudaMemcpyHostToDevice), "upload twiddles");
    if (rc == MHD_OK)
      rc = gcheck(g, cudaMemcpy((void*)(axis == 0 ? fp.ktx : fp.kty), k.data(), (size_t)n * 8,
                                cudaMemcpyHostToDevice), "upload wavenumbers");
  }
  const std::vector<int2> din = disk(gp->r_inner, dx, dy), dl = disk(gp->r_lane, dx, dy);
  std::vector<double2> wl(dl.size());
  for (size_t n = 0; n < dl.size(); ++n) {
    const double ex = dl[n].x * dx, ey = dl[n].y * dy;
    const double r = sqrt(ex * ex + ey * ey);
    double f;
    if (r <= gp->r_granule) {
      f = r / gp->r_granule;
    } else {
      const double c = cos(0.5 * M_PI * (r - gp->r_granule) / (gp->r_lane - gp->r_granule));
      f = c * c;
    }
    wl[n] = make_double2(f * ex / r, f * ey / r);
  }
  if (rc == MHD_OK && !din.empty())
    rc = gcheck(g, cudaMemcpy((void*)d.off_in, din.data(), din.size() * 8, cudaMemcpyHostToDevice), "upload disk");
  if (rc == MHD_OK)
    rc = gcheck(g, cudaMemcpy((void*)d.off_l, dl.data(), dl.size() * 8, cudaMemcpyHostToDevice), "upload lane");
  if (rc == MHD_OK)
    rc = gcheck(g, cudaMemcpy((void*)d.w_l, wl.data(), wl.size() * 16, cudaMemcpyHostToDevice), "upload weights");
  if (rc == MHD_OK)
    rc = gcheck(g, cudaMemsetAsync(g->ws + o.occ, 0, N * 4, g->st), "clear granules");
  if (rc == MHD_OK)
    rc = gcheck(g, cudaMemsetAsync(g->ws + o.par, 0, 4 * N * 8, g->st), "clear granules");
  if (rc == MHD_OK)
    rc = gcheck(g, cudaMemsetAsync(g->ws + o.vg, 0, 4 * N * 8, g->st), "clear fields");
  if (rc == MHD_OK) rc = gcheck(g, cudaStreamSynchronize(g->st), "create");
  if (rc != MHD_OK) {
    set_global_error("%s", g->err);
    delete g;
    return rc;
  }
  *out = g;
  return MHD_OK;
}

static const void* stage(mhd_gran_ctx* g, const void* src, size_t off, size_t bytes, int mem, int* rc) {
  if (mem == MHD_MEM_DEVICE) return src;
  *rc = gcheck(g, cudaMemcpyAsync(g->ws + off, src, bytes, cudaMemcpyHostToDevice, g->st), "stage input");
  return g->ws + off;
}

extern "C" int mhd_gran_update(mhd_gran_handle g, double t, const unsigned int* keys, const double* c_life,
                               const double* c_amp, int mem, int* rounds) {
  if (!g) return gfail(nullptr, MHD_ERR_ARG, "generator is NULL");
  if (!keys || !c_life || !c_amp) return gfail(g, MHD_ERR_ARG, "keys, c_life and c_amp are required");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return gfail(g, MHD_ERR_ARG, "bad mem flag");
  if (!std::isfinite(t)) return gfail(g, MHD_ERR_ARG, "t must be finite");
  const size_t N = (size_t)g->nx * g->ny;
  int rc = MHD_OK;
  const unsigned* k = (const unsigned*)stage(g, keys, g->o.keys, N * 4, mem, &rc);
  const double* cl = rc ? nullptr : (const double*)stage(g, c_life, g->o.cl, N * 8, mem, &rc);
  const double* ca = rc ? nullptr : (const double*)stage(g, c_amp, g->o.ca, N * 8, mem, &rc);
  if (rc) return rc;
  const int nb = g->o.nblk;
  expire_kernel<<<nb, GT, 0, g->st>>>(g->g, t);
  seed_kernel<<<nb, GT, 0, g->st>>>(g->g);
  g->launches += 2;
  // each round the first undecided pixel in (key, index) order joins, so
  // N + 1 rounds always suffice
  int r = 0, left = 1;
  while (left > 0) {
    if (r > (int)N) return gfail(g, MHD_ERR_TIMEOUT, "placement did not settle in %d rounds", r);
    rc = gcheck(g, cudaMemsetAsync(g->g.cnt, 0, 4, g->st), "clear count");
    if (rc) return rc;
    join_kernel<<<nb, GT, 0, g->st>>>(g->g, k);
    exclude_kernel<<<nb, GT, 0, g->st>>>(g->g);
    g->launches += 2;
    rc = gcheck(g, cudaMemcpyAsync(&left, g->g.cnt, 4, cudaMemcpyDeviceToHost, g->st), "read count");
    if (rc == MHD_OK) rc = gcheck(g, cudaStreamSynchronize(g->st), "placement round");
    if (rc) return rc;
    ++r;
  }
  birth_kernel<<<nb, GT, 0, g->st>>>(g->g, g->gp, t, cl, ca);
  g->launches += 1;
  if (rounds) *rounds = r;
  rc = gcheck(g, cudaGetLastError(), "update");
  if (rc == MHD_OK && mem == MHD_MEM_HOST) rc = gcheck(g, cudaStreamSynchronize(g->st), "update");
  return rc;
}

extern "C" int mhd_gran_velocity(mhd_gran_handle g, double t, int precision, void* v, int mem) {
  if (!g) return gfail(nullptr, MHD_ERR_ARG, "generator is NULL");
  if (!v) return gfail(g, MHD_ERR_ARG, "v is NULL");
  if (precision != 32 && precision != 64) return gfail(g, MHD_ERR_ARG, "precision must be 32 or 64");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return gfail(g, MHD_ERR_ARG, "bad mem flag");
  if (!std::isfinite(t)) return gfail(g, MHD_ERR_ARG, "t must be finite");
  const size_t N = (size_t)g->nx * g->ny;
  const int nb = g->o.nblk;
  const GranDev& d = g->g;
  amp_kernel<<<nb, GT, 0, g->st>>>(d, t);
  render_kernel<<<nb, GT, 0, g->st>>>(d);
  launch_rotational(g->fp, d.vg, d.vg + N, d.vr, d.vr + N, g->st);
  combine_kernel<<<nb, GT, 0, g->st>>>(d, g->gp.f_rot, nb);
  total_kernel<<<1, GT, 0, g->st>>>(d, nb);
  g->launches += 7;
  // device output straight into v; host output through the FFT's row
  // spectra (2N doubles), free once the column pass has read them
  void* dst = mem == MHD_MEM_DEVICE ? v : (void*)(g->ws + g->o.P);
  if (precision == 64) scale_kernel<double><<<nb, GT, 0, g->st>>>(d, (double*)dst);
  else scale_kernel<float><<<nb, GT, 0, g->st>>>(d, (float*)dst);
  g->launches += 1;
  int rc = gcheck(g, cudaGetLastError(), "velocity");
  if (rc == MHD_OK && mem == MHD_MEM_HOST) {
    rc = gcheck(g, cudaMemcpyAsync(v, dst, 2 * N * (precision == 64 ? 8 : 4), cudaMemcpyDeviceToHost, g->st),
                "read velocity");
    if (rc == MHD_OK) rc = gcheck(g, cudaStreamSynchronize(g->st), "read velocity");
  }
  return rc;
}

static int copy_out(mhd_gran_ctx* g, void* dst, const void* src, size_t bytes, int mem) {
  const cudaMemcpyKind kind = mem == MHD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int rc = gcheck(g, cudaMemcpyAsync(dst, src, bytes, kind, g->st), "read");
  if (rc == MHD_OK && mem == MHD_MEM_HOST) rc = gcheck(g, cudaStreamSynchronize(g->st), "read");
  return rc;
}

extern "C" int mhd_gran_read_granules(mhd_gran_handle g, int* occ, double* par, int mem) {
  if (!g) return gfail(nullptr, MHD_ERR_ARG, "generator is NULL");
  if (!occ) return gfail(g, MHD_ERR_ARG, "occ is NULL");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return gfail(g, MHD_ERR_ARG, "bad mem flag");
  const size_t N = (size_t)g->nx * g->ny;
  int rc = copy_out(g, occ, g->g.occ, N * 4, mem);
  if (rc == MHD_OK && par) rc = copy_out(g, par, g->g.t0, 4 * N * 8, mem);
  return rc;
}

extern "C" int mhd_gran_read_field(mhd_gran_handle g, int which, double* dst, int mem) {
  if (!g) return gfail(nullptr, MHD_ERR_ARG, "generator is NULL");
  if (!dst) return gfail(g, MHD_ERR_ARG, "dst is NULL");
  if (which != 0 && which != 1) return gfail(g, MHD_ERR_ARG, "which must be 0 or 1");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return gfail(g, MHD_ERR_ARG, "bad mem flag");
  const size_t N = (size_t)g->nx * g->ny;
  if (which == 0) return copy_out(g, dst, g->g.vg, 2 * N * 8, mem);
  // v_rot' is not kept (combine_kernel overwrites it with v_vor): recompute
  // it from v_gran into the FFT's row spectra, free once the column pass has
  // read them
  launch_rotational(g->fp, g->g.vg, g->g.vg + N, (double*)(g->ws + g->o.P), (double*)(g->ws + g->o.P) + N,
                    g->st);
  g->launches += 3;
  int rc = gcheck(g, cudaGetLastError(), "rotational part");
  if (rc) return rc;
  return copy_out(g, dst, g->ws + g->o.P, 2 * N * 8, mem);
}

extern "C" long long mhd_gran_launch_count(mhd_gran_handle g) { return g ? g->launches : 0; }

extern "C" const char* mhd_gran_last_error(mhd_gran_handle g) { return g ? g->err : mhd_last_error(nullptr); }

extern "C" void mhd_gran_destroy(mhd_gran_handle g) { delete g; }
