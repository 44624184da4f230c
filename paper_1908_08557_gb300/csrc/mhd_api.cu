// mhd_api.cu -- the C ABI of libmhd (declared in include/mhd.h): handle,
// workspace carving, host-built FFT tables, and the launch sequence of one RK3
// step.  All device memory comes from the caller's workspace.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/mhd.h"
#include "mhd_internal.h"

using namespace mhd;

struct mhd_ctx {
  CUtensorMap tm[3];   // TMA descriptors of the two FP32 state sets and of the adjoint's
                       // third substep state (64-byte aligned)
  CUtensorMap tma[2];  // the two state sets, boxes of A only (split pass A)
  CUtensorMap tmr[2];  // the two state sets, boxes of u, ln rho, ln T (split pass R)
  CUtensorMap tmdf;    // the RK accumulator, 32 x 8 tiles of the 8 fields (pair kernel)
  CUtensorMap tmdbar;  // its adjoint D, the same tiles (pair kernel, adjoint mode)
  bool tiled;          // FP32: TMA-fed z-march kernels; otherwise the simple kernel
  bool split;          // FP32 forward: split passes (else the fused z-march kernel)
  bool pair;           // FP32 forward: one-pass f32x2 kernel with TMEM z histories
  void* bj;            // split: [6][nz][ny][nx] B, J of the current substep
  void* sw;            // split: [3][nz - ksw][ny][nx] swamp terms
  int ksw;             // first layer with a nonzero swamp weight or slope (nz if none)
  bool adj_tiled;      // adjoint: tiled gather and (FP32) z-march point kernel, else one thread per point
  bool adj_zm;         // adjoint gather as a z-march (else 3D tiles after a grad-div fold)
  bool adj_pair;       // FP32 adjoint point kernel on the pair z-march (else the one-cell-per-thread z-march)
  mhd_params p;
  Layout L;
  cudaStream_t st;
  cudaStream_t side;   // highest-priority stream for the potential-field FFT of substep 0,
                       // forked from and joined to `st` by events (FFT boundary only)
  cudaEvent_t evf, evj;
  cudaEvent_t evc;     // end of the host-to-device driver copies (mhd_set_driver)
  PlaneStreams ps;     // two more FFT streams (planes 1, 2 of the potential-field boundary)
  size_t esz;          // bytes per state element
  char* ws;
  size_t ws_bytes;
  void* f[2];          // two state sets (ping-pong)
  void* df;            // RK accumulator (also interior pack scratch)
  int cur;
  void* lnrho0;        // [3] fixed density ghosts below the photosphere (state precision)
  void* wtab;          // [nz] swamp weight w(z_k)
  void* wptab;         // [nz] dw/dz
  void* bz;            // [ny][nx]
  void* axt;           // [ny][nx]
  void* ayt;
  void* v0;            // [2][ny][nx]
  void* v1;
  double* red;         // reduction partials
  double* cfl;         // CFL maxima slots [2 * CFL_SLOTS] (after the partials)
  StepState* ss;
  void* bgtab;         // background tables: lbar, tbar [nz+6]; dl, d2l, dt, d2t [nz]
  // adjoint buffers (params.adjoint)
  void* s2;            // third forward substep state
  void* fbar;          // state adjoint (padded)
  void* dbar;          // RK accumulator adjoint (padded)
  void* gbar;          // adjoint of the ghost-filled input of one RHS (padded)
  void* coef;          // [NCOEF_ADJ][nz][ny][nx] transposed-stencil coefficients
  double* thbar;       // [6][ny][nx] parameter adjoints (FP64)
  Background<float> bgf;
  Background<double> bgd;
  // A stored about a fixed FP64 background (params a_background)
  bool abg_mode;
  void* abB;           // [6][nz][ny][nx]: B_bg (3), J_bg (3), state precision
  void* abL;           // [4][nz - ksw][ny][nx]: lap A_bg (3), div A_bg on the swamp layers
  void* abgR;          // A_bg in the padded layout, fields 0..2, state precision
  double* abg0;        // [2][ny][nx] FP64 A_bg_x, A_bg_y at the photosphere
  double* at64;        // [3][ny][nx] FP64 scratch: B_z target, A_x, A_y of the target
  void* atrel;         // [2][ny][nx] nudging target minus A_bg(k = 0), state precision
  // non-uniform vertical grid (params z): the handle's copy of the positions
  // (p.z points here), and the device tables dxi/dz, (d2xi/dz2)/(dxi/dz),
  // z_k, cell extent, [4][nz] in the state precision
  double* zh;
  void* ztab;
  double* zt64;        // [2][nz] FP64 dxi/dz and r21 (the background tables' stencils)
  FFTPlan fp;
  bool have_fft;
  bool driver_set;
  double t0, t1;
  long long host_steps;
  long long nlaunch;                  // kernels launched since create
  bool prof;                          // bracket kernel classes with events
  bool serial;                        // profiling with every kernel on the handle's stream, one after another
  int dbg_skip_plane;                 // time-out test hook for the next forward FP32 launch (INT_MIN: off)
  int dbg_wait_limit;
  struct Ev { cudaEvent_t a, b; int cls; int nk; };
  std::vector<Ev>* evs;
  char err[512];
};

// bracket one kernel class launch (nk kernels) with events when profiling
struct ClassTimer {
  mhd_ctx* h;
  mhd_ctx::Ev ev;
  cudaStream_t st;
  ClassTimer(mhd_ctx* h_, int cls, int nk, cudaStream_t s = nullptr) : h(h_), st(s ? s : h_->st) {
    h->nlaunch += nk;
    ev.cls = cls;
    ev.nk = nk;
    if (h->prof) {
      cudaEventCreate(&ev.a);
      cudaEventCreate(&ev.b);
      cudaEventRecord(ev.a, st);
    }
  }
  ~ClassTimer() {
    if (h->prof) {
      cudaEventRecord(ev.b, st);
      h->evs->push_back(ev);
    }
  }
};

static char g_err[512] = "no error";

static int fail(mhd_ctx* h, int code, const char* fmt, ...) {
  char* buf = h ? h->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return code;
}

// message for mhd_last_error(NULL), used by entry points without a handle
void mhd::set_global_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

static int cuda_check(mhd_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, MHD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return MHD_OK;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// position of layer k (-3 .. nz + 2): the given vertical grid, or k dz
static double zpos(const mhd_params* p, int k) { return p->z ? p->z[k + NG] : (double)k * p->dz; }

// sixth-order index-space derivatives of the positions at an interior layer:
// dz/dxi and d2z/dxi2 (dz and 0 on the uniform grid)
static void zderiv(const mhd_params* p, int k, double* z1, double* z2) {
  static const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
  static const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0, 2.0 / 180.0};
  if (!p->z) {
    *z1 = p->dz;
    *z2 = 0.0;
    return;
  }
  double a = 0.0, b = W2[0] * zpos(p, k);
  for (int m = 1; m <= 3; ++m) {
    a += W1[m] * (zpos(p, k + m) - zpos(p, k - m));
    b += W2[m] * (zpos(p, k + m) + zpos(p, k - m));
  }
  *z1 = a;
  *z2 = b;
}
static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

static const char* check_params(const mhd_params* p) {
  if (!p) return "params is NULL";
  if (p->precision != 32 && p->precision != 64) return "precision must be 32 or 64";
  if (p->nx < 4 || p->ny < 4) return "nx, ny must be >= 4";
  if (p->nz < 7) return "nz must be >= 7";
  if (p->bc_z != 0 && p->bc_z != 1) return "bc_z must be 0 or 1";
  if (p->bc_z == 0) {
    if (!is_pow2(p->nx) || !is_pow2(p->ny) || p->nx < 8 || p->ny < 8 || p->nx > 1024 || p->ny > 1024)
      return "with bc_z = 0, nx and ny must be powers of two in [8, 1024]";
  }
  if (!(p->dx > 0) || !(p->dy > 0) || !(p->dz > 0)) return "grid spacings must be positive";
  if (!(p->gamma > 1.0)) return "gamma must exceed 1";
  if (p->stats_every < 0) return "stats_every must be >= 0";
  if (p->adjoint != 0 && p->adjoint != 1) return "adjoint must be 0 or 1";
  if (p->a_background != 0 && p->a_background != 1) return "a_background must be 0 or 1";
  if (p->a_background && p->adjoint) return "a_background is not supported with adjoint = 1";
  if (p->z) {
    if (p->adjoint) return "a non-uniform vertical grid is not supported with adjoint = 1";
    for (int q = 0; q + 1 < p->nz + 2 * NG; ++q)
      if (!(p->z[q + 1] > p->z[q])) return "z: the nz + 6 layer positions must increase strictly";
    for (int k = 0; k < p->nz; ++k) {
      double z1, z2;
      zderiv(p, k, &z1, &z2);
      if (!(z1 > 0.0)) return "z: the sixth-order dz/dxi must be positive at every interior layer";
    }
  }
  if ((long long)p->nx * p->ny * p->nz > (1LL << 34)) return "grid too large";
  if (p->adjoint && (long long)NF * (p->nz + 2 * NG) * p->ny * (p->nx / 4) >= (1LL << 31))
    return "grid too large for the adjoint (8 (nz + 6) ny nx / 4 must stay below 2^31)";
  if ((long long)((p->nx + 31) / 32) * ((p->ny + 7) / 8) > RED_BLOCKS_MAX)
    return "horizontal grid too large for the reduction buffer (nx * ny <= 2^20)";
  if (!(p->nc_tau >= 0.0)) return "nc_tau must be >= 0";
  if (p->nc_tau > 0.0 && !(p->nc_lnrho_width > 0.0 && p->nc_lnrho_width <= p->nc_lnrho_magn && p->nc_z_width > 0.0))
    return "Newtonian cooling needs 0 < nc_lnrho_width <= nc_lnrho_magn and nc_z_width > 0";
  return nullptr;
}

// ---- workspace carving ------------------------------------------------------
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

struct Offsets {
  size_t f0, f1, df, lnrho0, wtab, wptab, bz, axt, ayt, v0, v1, red, ss, bg, bj, sw;
  size_t s2, fbar, dbar, gbar, coef, thbar;
  size_t abB, abL, abgR, abg0, at64, atrel, ztab, zt64;
  size_t twx, twy, et, eb, ktx, kty, P, Q;
  size_t total;
};

static void swamp_weight(const mhd_params* p, double z, double* w, double* wp);

// first layer whose swamp weight or slope is nonzero (nz if none)
static int swamp_first_layer(const mhd_params* p) {
  for (int k = 0; k < p->nz; ++k) {
    double w, wp;
    swamp_weight(p, zpos(p, k), &w, &wp);
    if (w != 0.0 || wp != 0.0) return k;
  }
  return p->nz;
}

static Offsets plan_offsets(const mhd_params* p) {
  Offsets o;
  Carve c;
  Layout L = make_layout(p->nx, p->ny, p->nz);
  size_t es = p->precision == 64 ? 8 : 4;
  size_t set = (size_t)NF * L.fs * es;
  size_t n2 = (size_t)p->nx * p->ny;
  o.f0 = c.take(set);
  o.f1 = c.take(set);
  o.df = c.take(set);
  o.lnrho0 = c.take(8 * es);
  o.wtab = c.take((size_t)p->nz * es);
  o.wptab = c.take((size_t)p->nz * es);
  o.bz = c.take(n2 * es);
  o.axt = c.take(n2 * es);
  o.ayt = c.take(n2 * es);
  o.v0 = c.take(2 * n2 * es);
  o.v1 = c.take(2 * n2 * es);
  o.red = c.take(((size_t)RED_BLOCKS_MAX * 8 + 2 * CFL_SLOTS) * sizeof(double));
  o.ss = c.take(sizeof(StepState));
  o.bg = c.take((size_t)(6 * p->nz + 12) * es);
  o.ztab = c.take((size_t)4 * p->nz * es);
  o.zt64 = c.take((size_t)2 * p->nz * 8);
  if (p->precision == 32 && !p->a_background) {
    o.bj = c.take((size_t)6 * n2 * p->nz * 4);
    o.sw = c.take((size_t)3 * n2 * (p->nz - swamp_first_layer(p)) * 4);
  } else {
    o.bj = o.sw = 0;
  }
  if (p->a_background) {
    o.abB = c.take((size_t)6 * n2 * p->nz * es);
    o.abL = c.take((size_t)4 * n2 * (p->nz - swamp_first_layer(p)) * es);
    o.abgR = c.take((size_t)3 * L.fs * es);
    o.abg0 = c.take(2 * n2 * 8);
    o.at64 = c.take(3 * n2 * 8);
    o.atrel = c.take(2 * n2 * es);
  } else {
    o.abB = o.abL = o.abgR = o.abg0 = o.at64 = o.atrel = 0;
  }
  if (p->adjoint) {
    o.s2 = c.take(set);
    o.fbar = c.take(set);
    o.dbar = c.take(set);
    o.gbar = c.take(set);
    o.coef = c.take((size_t)NCOEF_ADJ * p->nx * p->ny * p->nz * es);
    o.thbar = c.take(6 * n2 * sizeof(double));
  } else {
    o.s2 = o.fbar = o.dbar = o.gbar = o.coef = o.thbar = 0;
  }
  if (p->bc_z == 0) {
    o.twx = c.take((size_t)p->nx * 16);
    o.twy = c.take((size_t)p->ny * 16);
    o.et = c.take(3 * n2 * 8);
    o.eb = c.take(3 * n2 * 8);
    o.ktx = c.take((size_t)p->nx * 8);
    o.kty = c.take((size_t)p->ny * 8);
    o.P = c.take(3 * n2 * 16);
    o.Q = c.take(9 * n2 * 16);
  } else {
    o.twx = o.twy = o.et = o.eb = o.ktx = o.kty = o.P = o.Q = 0;
  }
  o.total = c.off;
  return o;
}

extern "C" size_t mhd_workspace_bytes(const mhd_params* p) {
  if (check_params(p)) return 0;
  return plan_offsets(p).total;
}

// ---- helpers ----------------------------------------------------------------
template <typename R>
static Phys<R> make_phys(const mhd_params* p) {
  Phys<R> ph;
  ph.idx = (R)(1.0 / p->dx);
  ph.idy = (R)(1.0 / p->dy);
  ph.idz = (R)(1.0 / p->dz);
  ph.idx2 = (R)(1.0 / (p->dx * p->dx));
  ph.idy2 = (R)(1.0 / (p->dy * p->dy));
  ph.idz2 = (R)(1.0 / (p->dz * p->dz));
  ph.gamma = (R)p->gamma;
  ph.gm1 = (R)(p->gamma - 1.0);
  ph.gz = (R)p->gz;
  ph.nu = (R)p->nu;
  ph.eta = (R)p->eta;
  ph.kappa0 = (R)p->kappa0;
  ph.drho = (R)p->diff_rho;
  ph.eta_s = (R)p->eta_swamp;
  ph.chi_s = (R)p->chi_swamp;
  ph.drho_s = (R)p->diffrho_swamp;
  ph.tau_u = (R)p->tau_u;
  ph.tau_A = (R)p->tau_A;
  for (int c = 0; c < 3; ++c) ph.bext[c] = (R)p->bext[c];
  ph.bcz = p->bc_z;
  ph.nc_tau = (R)p->nc_tau;
  ph.nc_lmag = (R)p->nc_lnrho_magn;
  ph.nc_lw = (R)p->nc_lnrho_width;
  ph.nc_zmax = (R)p->nc_z_max;
  ph.nc_zw = (R)p->nc_z_width;
  ph.dz = (R)p->dz;
  // layers below the height cut-off (c_z(k dz) > 0); none when off
  ph.nc_k1 = 0;
  if (p->nc_tau > 0.0 && p->bc_z == 0)
    while (ph.nc_k1 < p->nz && zpos(p, ph.nc_k1) < p->nc_z_max) ++ph.nc_k1;
  return ph;
}

// cubic swamp weight (Sect. 4.3): 0 below z_s, 1 above z_t, zero end slopes
static void swamp_weight(const mhd_params* p, double z, double* w, double* wp) {
  double zs = p->z_swamp_start, zt = p->z_swamp_end;
  *w = 0.0;
  *wp = 0.0;
  if (!(zt > zs)) return;
  double s = (z - zs) / (zt - zs);
  if (s <= 0.0) return;
  if (s >= 1.0) { *w = 1.0; return; }
  *w = s * s * (3.0 - 2.0 * s);
  *wp = 6.0 * s * (1.0 - s) / (zt - zs);
}

static void driver_weights(const mhd_ctx* h, double t, double* r, double* s) {
  *r = 1.0;
  if (h->p.t_ramp > 0.0) *r = fmin(fmax(t / h->p.t_ramp, 0.0), 1.0);
  double q = h->t1 > h->t0 ? (t - h->t0) / (h->t1 - h->t0) : 0.0;
  *s = fmin(fmax(q, 0.0), 1.0);
}

static cudaMemcpyKind kind_in(int mem) { return mem == MHD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
static cudaMemcpyKind kind_out(int mem) { return mem == MHD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

static int sync_status(mhd_ctx* h) {
  int rc = cuda_check(h, cudaStreamSynchronize(h->st), "stream synchronize");
  if (rc) return rc;
  int nf = 0;
  rc = cuda_check(h, cudaMemcpy(&nf, &h->ss->nonfinite, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (rc) return rc;
  if (nf) return fail(h, MHD_ERR_NONFINITE, "non-finite value in the state (time stepping halted)");
  return MHD_OK;
}

template <typename R> static const Background<R>& bgr(const mhd_ctx* h);
template <> const Background<float>& bgr<float>(const mhd_ctx* h) { return h->bgf; }
template <> const Background<double>& bgr<double>(const mhd_ctx* h) { return h->bgd; }

// Background profiles of ln rho and ln T (FP64): the given initial profiles
// (ln T: horizontal means of the initial state when no profile is given),
// their sixth-order z derivatives at interior layers, and the constants the
// ghost rules need in perturbation form.  Zero in the periodic-z geometry.
template <typename R>
static int upload_background(mhd_ctx* h, const double* lnrho0, const double* lnT0, const double* tmean) {
  const mhd_params* p = &h->p;
  const int nz = p->nz, n6 = nz + 2 * NG, kt = nz - 1;
  std::vector<double> lb(n6, 0.0), tb(n6, 0.0);
  if (p->bc_z == 0) {
    for (int q = 0; q < n6; ++q) lb[q] = lnrho0[q];
    if (lnT0) {
      for (int q = 0; q < n6; ++q) tb[q] = lnT0[q];
    } else {
      for (int k = 0; k < nz; ++k) tb[k + NG] = tmean[k];
      for (int m = 1; m <= NG; ++m) {
        const int b1 = NG - m + 1, b0 = NG - m;
        const double dzm = zpos(p, 1 - m) - zpos(p, -m);
        tb[b0] = tb[b1] + lb[b1] - lb[b0] - dzm * p->gz / exp(tb[b1]);
        tb[NG + kt + m] = tb[NG + kt - m];
      }
    }
  }
  static const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
  static const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0, 2.0 / 180.0};
  std::vector<R> tab((size_t)6 * nz + 12, R(0));
  R* t_lb = tab.data();
  R* t_tb = t_lb + n6;
  R* t_dl = t_tb + n6;
  R* t_d2l = t_dl + nz;
  R* t_dt = t_d2l + nz;
  R* t_d2t = t_dt + nz;
  for (int q = 0; q < n6; ++q) { t_lb[q] = (R)lb[q]; t_tb[q] = (R)tb[q]; }
  for (int k = 0; k < nz; ++k) {
    const int c = k + NG;
    double a1 = 0, a2 = W2[0] * lb[c], b1 = 0, b2 = W2[0] * tb[c];
    for (int m = 1; m <= 3; ++m) {
      a1 += W1[m] * (lb[c + m] - lb[c - m]);
      a2 += W2[m] * (lb[c + m] + lb[c - m]);
      b1 += W1[m] * (tb[c + m] - tb[c - m]);
      b2 += W2[m] * (tb[c + m] + tb[c - m]);
    }
    if (p->z) {
      // chain rule: D_z f = f_xi / z', D_z^2 f = f_xixi / z'^2 - f_xi z'' / z'^3
      double z1, z2;
      zderiv(p, k, &z1, &z2);
      t_dl[k] = (R)(a1 / z1);
      t_d2l[k] = (R)(a2 / (z1 * z1) - a1 * z2 / (z1 * z1 * z1));
      t_dt[k] = (R)(b1 / z1);
      t_d2t[k] = (R)(b2 / (z1 * z1) - b1 * z2 / (z1 * z1 * z1));
    } else {
      t_dl[k] = (R)(a1 / p->dz);
      t_d2l[k] = (R)(a2 / (p->dz * p->dz));
      t_dt[k] = (R)(b1 / p->dz);
      t_d2t[k] = (R)(b2 / (p->dz * p->dz));
    }
  }
  Background<R> bg;
  bg.lbar = (const R*)h->bgtab;
  bg.tbar = bg.lbar + n6;
  bg.dl = bg.tbar + n6;
  bg.d2l = bg.dl + nz;
  bg.dt = bg.d2l + nz;
  bg.d2t = bg.dt + nz;
  for (int m = 0; m <= NG; ++m) { bg.cb[m] = R(0); bg.ctT[m] = R(0); bg.ctL[m] = R(0); }
  bg.ksw = h->ksw;
  bg.bB = bg.bJ = bg.bL = bg.abg = nullptr;
  // vertical grid: ghost-rule distances, and the per-layer tables
  for (int m = 0; m <= NG; ++m) { bg.dzb[m] = R(0); bg.dzt[m] = R(0); }
  for (int m = 1; m <= NG; ++m) {
    bg.dzb[m] = (R)(zpos(p, 1 - m) - zpos(p, -m));
    bg.dzt[m] = (R)(zpos(p, kt + m) - zpos(p, kt - m));
  }
  bg.zm1 = bg.zr21 = bg.zk = bg.zcell = nullptr;
  if (p->z) {
    std::vector<R> zt((size_t)4 * nz);
    std::vector<double> z64((size_t)2 * nz);
    for (int k = 0; k < nz; ++k) {
      double z1, z2;
      zderiv(p, k, &z1, &z2);
      zt[k] = (R)(1.0 / z1);
      zt[(size_t)nz + k] = (R)(-z2 / (z1 * z1));
      zt[(size_t)2 * nz + k] = (R)zpos(p, k);
      zt[(size_t)3 * nz + k] = (R)(0.5 * (zpos(p, k + 1) - zpos(p, k - 1)));
      z64[k] = 1.0 / z1;
      z64[(size_t)nz + k] = -z2 / (z1 * z1);
    }
    int rz = cuda_check(h, cudaMemcpy(h->ztab, zt.data(), zt.size() * sizeof(R), cudaMemcpyHostToDevice),
                        "upload vertical grid");
    if (!rz) rz = cuda_check(h, cudaMemcpy(h->zt64, z64.data(), z64.size() * 8, cudaMemcpyHostToDevice),
                             "upload vertical grid (FP64)");
    if (rz) return rz;
    bg.zm1 = (const R*)h->ztab;
    bg.zr21 = bg.zm1 + nz;
    bg.zk = bg.zm1 + 2 * nz;
    bg.zcell = bg.zm1 + 3 * nz;
  }
  if (h->abg_mode) {
    const long long n3 = (long long)p->nx * p->ny * nz;
    bg.bB = (const R*)h->abB;
    bg.bJ = bg.bB + 3 * n3;
    bg.bL = (const R*)h->abL;
    bg.abg = (const R*)h->abgR;
  }
  for (int m = 1; m <= NG; ++m) {
    const int b1 = NG - m + 1, b0 = NG - m;
    bg.cb[m] = (R)(tb[b1] - tb[b0] + lb[b1] - lb[b0]);
    bg.ctT[m] = (R)(tb[NG + kt - m] - tb[NG + kt + m]);
    bg.ctL[m] = (R)(lb[NG + kt - m] - lb[NG + kt + m]);
  }
  if (sizeof(R) == 8) h->bgd = *(Background<double>*)&bg; else h->bgf = *(Background<float>*)&bg;
  return cuda_check(h, cudaMemcpy(h->bgtab, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice),
                    "upload background");
}

// ---- launch sequence ----------------------------------------------------------
template <typename R>
static void ghost_fill(mhd_ctx* h, R* f) {
  Phys<R> ph = make_phys<R>(&h->p);
  {
    ClassTimer ct(h, MHD_KC_GHOST, 1);
    launch_bc<R>(h->L, ph, bgr<R>(h), f, (R)h->p.dz, h->ss, h->st);
  }
  if (h->p.bc_z == 0) {
    ClassTimer ct(h, MHD_KC_PFE, 3);
    launch_pfe<R>(h->fp, h->L, f, h->ss, h->st, h->serial ? nullptr : &h->ps);
  }
}

static void release_side(mhd_ctx* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->ps.s[i]) {
      cudaStreamSynchronize(h->ps.s[i]);
      cudaStreamDestroy(h->ps.s[i]);
    }
    if (h->ps.join[i]) cudaEventDestroy(h->ps.join[i]);
    h->ps.s[i] = nullptr;
    h->ps.join[i] = nullptr;
  }
  if (h->ps.fork) cudaEventDestroy(h->ps.fork);
  h->ps.fork = nullptr;
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->evf) cudaEventDestroy(h->evf);
  if (h->evj) cudaEventDestroy(h->evj);
  if (h->evc) cudaEventDestroy(h->evc);
  if (h->side) cudaStreamDestroy(h->side);
  h->evf = h->evj = h->evc = nullptr;
  h->side = nullptr;
}

// sum of the inverse squared spacings of the CFL rule; with a non-uniform
// vertical grid the reduction applies each layer's own sum (this is then 1)
static double inv2sum(const mhd_params* p) {
  if (p->z) return 1.0;
  return 1.0 / (p->dx * p->dx) + 1.0 / (p->dy * p->dy) + 1.0 / (p->dz * p->dz);
}

template <typename R>
static void run_stats(mhd_ctx* h, R* f) {
  Phys<R> ph = make_phys<R>(&h->p);
  ClassTimer ct(h, MHD_KC_STATS, 3);
  // B into the RK accumulator: free here (substep 0 does not read it)
  int nb = launch_stats_partial<R>(h->L, ph, bgr<R>(h), f, (R*)h->df, h->red, h->st);
  // cell volume dx dy dz; with a non-uniform vertical grid each cell's
  // extent is applied in the partial sums
  const double dv = h->p.dx * h->p.dy * (h->p.z ? 1.0 : h->p.dz);
  launch_stats_finalize(h->red, nb, h->ss, dv, h->p.dx * h->p.dy, h->p.gamma - 1.0, h->st);
}

// fused RHS + RK launch: TMA-fed z-march for FP32 (unless disabled), the
// simple one-thread-per-cell kernel otherwise
// the nudging target the kernels see: A_target itself, or (A stored about a
// background) A_target - A_bg(k = 0), formed in FP64
static Driver kernel_driver(const mhd_ctx* h) {
  if (h->abg_mode)
    return Driver{h->atrel, (const char*)h->atrel + (size_t)h->p.nx * h->p.ny * h->esz, h->v0, h->v1};
  return Driver{h->axt, h->ayt, h->v0, h->v1};
}

// tmin: the tensor map of fin when fin is not one of the handle's two state
// sets (a tape of substep states)
template <typename R>
static void launch_rk_any(mhd_ctx* h, const R* fin, R* fout, int sub, const CUtensorMap* tmin = nullptr) {
  Phys<R> ph = make_phys<R>(&h->p);
  Driver drv = kernel_driver(h);
  if (sizeof(R) == 4 && h->pair) {
    const int which = (const void*)fin == h->f[0] ? 0 : 1;
    // on a non-uniform vertical grid the z stencils run in index space
    // (unit spacing) and the kernel applies the metric per layer
    launch_rk_pair(tmin ? tmin : &h->tm[which], &h->tmdf, h->L, *(const Phys<float>*)&ph, h->bgf, (float*)fout, (float*)h->df,
                   (const float*)h->wtab, (const float*)h->wptab, drv, h->ss, sub, h->p.dx, h->p.dy,
                   h->p.z ? 1.0 : h->p.dz, h->st, h->dbg_skip_plane, h->dbg_wait_limit);
    h->dbg_skip_plane = INT_MIN;  // one launch only
    return;
  }
  if (sizeof(R) == 4 && h->split) {
    const int which = (const void*)fin == h->f[0] ? 0 : 1;
    launch_rk_split(&h->tma[which], &h->tmr[which], h->L, *(const Phys<float>*)&ph, h->bgf, (const float*)fin,
                    (float*)fout, (float*)h->df, (float*)h->bj, (float*)h->sw, h->ksw, (const float*)h->wtab,
                    (const float*)h->wptab, drv, h->ss, sub, h->p.dx, h->p.dy, h->p.dz, h->st);
    return;
  }
  if (sizeof(R) == 4 && h->tiled) {
    const int which = (const void*)fin == h->f[0] ? 0 : 1;
    launch_rk_tiled(&h->tm[which], h->L, *(const Phys<float>*)&ph, h->bgf, (float*)fout, (float*)h->df,
                    (const float*)h->wtab, (const float*)h->wptab, drv, h->ss, sub, h->p.dx, h->p.dy, h->p.dz,
                    h->st);
    return;
  }
  launch_rk<R>(h->L, ph, bgr<R>(h), fin, fout, (R*)h->df, (const R*)h->wtab, (const R*)h->wptab, drv, h->ss, sub,
               h->st);
}

// CFL maxima over the inner layers (k = 3 .. nz - 4) of fin: the z-march
// kernel for the FP32 state sets, else the plane-parallel one
template <typename R>
static void cfl_inner(mhd_ctx* h, const R* fin, bool zero) {
  Phys<R> ph = make_phys<R>(&h->p);
  if (sizeof(R) == 4 && h->pair && ((const void*)fin == h->f[0] || (const void*)fin == h->f[1])) {
    const int which = (const void*)fin == h->f[0] ? 0 : 1;
    launch_cfl_inner_zm(&h->tma[which], h->L, *(const Phys<float>*)&ph, h->bgf, (const float*)fin,
                        (const float*)h->wtab, h->cfl, h->ss, zero, h->st);
    return;
  }
  launch_cfl_partial<R>(h->L, ph, bgr<R>(h), fin, (const R*)h->wtab, h->cfl, h->ss, CflPlanes::inner, zero, h->st);
}

template <typename R>
static void run_step(mhd_ctx* h, bool stats) {
  Phys<R> ph = make_phys<R>(&h->p);
  for (int sub = 0; sub < 3; ++sub) {
    R* fin = (R*)h->f[h->cur];
    R* fout = (R*)h->f[1 - h->cur];
    const bool adaptive = !(h->p.dt_fixed > 0.0);
    if (sub == 0 && adaptive && h->side && !h->serial && h->L.nz > 2 * NG) {
      // The FFT of the potential-field ghosts (FP64-pipe bound) runs on the
      // side stream while the ghost rules and the CFL reduction over the
      // inner layers (whose stencils read no ghost plane) run here; the
      // three layers at each end follow once the FFT has joined.  Neither
      // side writes what the other reads: the FFT writes only the A ghost
      // planes, the ghost rules only those of u, ln rho, ln T.
      cudaEventRecord(h->evf, h->st);
      cudaStreamWaitEvent(h->side, h->evf, 0);
      {
        ClassTimer ct(h, MHD_KC_PFE, 3, h->side);
        launch_pfe<R>(h->fp, h->L, fin, h->ss, h->side, &h->ps);
      }
      cudaEventRecord(h->evj, h->side);
      {
        ClassTimer ct(h, MHD_KC_GHOST, 1);
        launch_bc<R>(h->L, ph, bgr<R>(h), fin, (R)h->p.dz, h->ss, h->st);
      }
      {
        ClassTimer ct(h, MHD_KC_CFL, 1);
        cfl_inner<R>(h, fin, true);
      }
      cudaStreamWaitEvent(h->st, h->evj, 0);
      if (stats) run_stats<R>(h, fin);
      ClassTimer ct(h, MHD_KC_CFL, 2);
      int nb = launch_cfl_partial<R>(h->L, ph, bgr<R>(h), fin, (const R*)h->wtab, h->cfl, h->ss, CflPlanes::ends,
                                     false, h->st);
      launch_cfl_finalize(h->cfl, nb, h->ss, h->p.c_adv, h->p.c_diff, h->p.dt_fixed, inv2sum(&h->p), h->t0,
                          h->t1, h->p.t_ramp, 0, h->st);
    } else {
      ghost_fill<R>(h, fin);
      if (sub == 0) {
        if (stats) run_stats<R>(h, fin);
        const bool zmarch = adaptive && sizeof(R) == 4 && h->pair && h->L.nz > 2 * NG;
        ClassTimer ct(h, MHD_KC_CFL, zmarch ? 3 : (adaptive ? 2 : 1));
        int nb = 0;
        if (zmarch) {
          cfl_inner<R>(h, fin, true);
          nb = launch_cfl_partial<R>(h->L, ph, bgr<R>(h), fin, (const R*)h->wtab, h->cfl, h->ss, CflPlanes::ends,
                                     false, h->st);
        } else if (adaptive) {
          nb = launch_cfl_partial<R>(h->L, ph, bgr<R>(h), fin, (const R*)h->wtab, h->cfl, h->ss, CflPlanes::all,
                                     true, h->st);
        }
        launch_cfl_finalize(h->cfl, nb, h->ss, h->p.c_adv, h->p.c_diff, h->p.dt_fixed, inv2sum(&h->p), h->t0,
                            h->t1, h->p.t_ramp, 0, h->st);
      }
    }
    {
      ClassTimer ct(h, MHD_KC_RK, 1);
      launch_rk_any<R>(h, fin, fout, sub);
    }
    h->cur = 1 - h->cur;
  }
}

// ---- FFT tables (host, FP64) ----------------------------------------------------
static int upload_fft_tables(mhd_ctx* h, const Offsets& o) {
  const mhd_params* p = &h->p;
  int nx = p->nx, ny = p->ny;
  std::vector<double> tw((size_t)2 * (nx > ny ? nx : ny));
  FFTPlan& fp = h->fp;
  fp.nx = nx;
  fp.ny = ny;
  fp.lognx = ilog2(nx);
  fp.logny = ilog2(ny);
  fp.twx = (const double2*)(h->ws + o.twx);
  fp.twy = (const double2*)(h->ws + o.twy);
  fp.et = (const double*)(h->ws + o.et);
  fp.eb = (const double*)(h->ws + o.eb);
  fp.ktx = (const double*)(h->ws + o.ktx);
  fp.kty = (const double*)(h->ws + o.kty);
  fp.P = (double2*)(h->ws + o.P);
  fp.Q = (double2*)(h->ws + o.Q);
  int rc;
  for (int axis = 0; axis < 2; ++axis) {
    int n = axis == 0 ? nx : ny;
    for (int r = 0; r < n; ++r) {
      tw[2 * r] = cos(2.0 * M_PI * r / n);
      tw[2 * r + 1] = -sin(2.0 * M_PI * r / n);
    }
    rc = cuda_check(h, cudaMemcpy((void*)(axis == 0 ? fp.twx : fp.twy), tw.data(), (size_t)n * 16,
                                  cudaMemcpyHostToDevice), "upload twiddles");
    if (rc) return rc;
  }
  // continuous |k| = 2 pi sqrt((m/Lx)^2 + (n/Ly)^2), signed m, n; tables
  // [m - 1][kx][ky] for ghost layer m: exp(-|k| d_m) above the top layer,
  // d_m = z_{nz-1+m} - z_{nz-1} (Eq. 17), and exp(f_b |k| d'_m) below the
  // photosphere, d'_m = z_0 - z_{-m} (m dz on the uniform grid)
  double lx = nx * p->dx, ly = ny * p->dy;
  const size_t n2 = (size_t)nx * ny;
  std::vector<double> et(3 * n2), eb(3 * n2);
  const int kt = p->nz - 1;
  for (int m = 1; m <= NG; ++m) {
    const double dt = zpos(p, kt + m) - zpos(p, kt), db = zpos(p, 0) - zpos(p, -m);
    for (int a = 0; a < nx; ++a) {
      int ma = 2 * a > nx ? a - nx : a;
      double kx = 2.0 * M_PI * ma / lx;
      for (int b = 0; b < ny; ++b) {
        int mb = 2 * b > ny ? b - ny : b;
        double ky = 2.0 * M_PI * mb / ly;
        double kk = sqrt(kx * kx + ky * ky);
        et[(size_t)(m - 1) * n2 + (size_t)a * ny + b] = exp(-kk * dt);
        eb[(size_t)(m - 1) * n2 + (size_t)a * ny + b] = exp(p->f_pfe_bottom * kk * db);
      }
    }
  }
  rc = cuda_check(h, cudaMemcpy((void*)fp.et, et.data(), et.size() * 8, cudaMemcpyHostToDevice), "upload et");
  if (rc) return rc;
  rc = cuda_check(h, cudaMemcpy((void*)fp.eb, eb.data(), eb.size() * 8, cudaMemcpyHostToDevice), "upload eb");
  if (rc) return rc;
  // modified wavenumber of the sixth-order first derivative; zero at m = 0
  // and at the Nyquist mode
  for (int axis = 0; axis < 2; ++axis) {
    int n = axis == 0 ? nx : ny;
    double hsp = axis == 0 ? p->dx : p->dy;
    std::vector<double> kt((size_t)n);
    for (int m = 0; m < n; ++m) {
      if (m == 0 || 2 * m == n) { kt[m] = 0.0; continue; }
      double th = 2.0 * M_PI * (2 * m > n ? m - n : m) / n;
      kt[m] = (45.0 * sin(th) - 9.0 * sin(2.0 * th) + sin(3.0 * th)) / (30.0 * hsp);
    }
    rc = cuda_check(h, cudaMemcpy((void*)(axis == 0 ? fp.ktx : fp.kty), kt.data(), (size_t)n * 8,
                                  cudaMemcpyHostToDevice), "upload kt");
    if (rc) return rc;
  }
  return MHD_OK;
}

// ---- entry points --------------------------------------------------------------
extern "C" int mhd_create(const mhd_params* p, void* workspace, size_t ws_bytes, const void* init_state,
                          int mem, const double* lnrho0, const double* lnT0, void* stream, mhd_handle* out) {
  if (!out) return fail(nullptr, MHD_ERR_ARG, "out is NULL");
  *out = nullptr;
  const char* bad = check_params(p);
  if (bad) return fail(nullptr, MHD_ERR_ARG, "%s", bad);
  if (!init_state || !lnrho0) return fail(nullptr, MHD_ERR_ARG, "init_state and lnrho0 are required");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(nullptr, MHD_ERR_ARG, "bad mem flag");
  if (p->nc_tau > 0.0)
    for (int k = 0; k + 1 < p->nz; ++k)
      if (!(lnrho0[NG + k + 1] < lnrho0[NG + k]))
        return fail(nullptr, MHD_ERR_ARG, "Newtonian cooling needs ln rho0 falling strictly with height");
  Offsets o = plan_offsets(p);
  if (!workspace) return fail(nullptr, MHD_ERR_WORKSPACE, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(nullptr, MHD_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (ws_bytes < o.total)
    return fail(nullptr, MHD_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", ws_bytes, o.total);

  void* mem_ctx = nullptr;
  if (posix_memalign(&mem_ctx, 64, sizeof(mhd_ctx)) != 0 || !mem_ctx)
    return fail(nullptr, MHD_ERR_ARG, "host allocation failed");
  memset(mem_ctx, 0, sizeof(mhd_ctx));
  mhd_ctx* h = (mhd_ctx*)mem_ctx;
  h->p = *p;
  if (p->z) {
    // the handle keeps its own copy of the vertical grid
    h->zh = (double*)malloc(sizeof(double) * (size_t)(p->nz + 2 * NG));
    if (!h->zh) {
      free(h);
      return fail(nullptr, MHD_ERR_ARG, "host allocation failed");
    }
    memcpy(h->zh, p->z, sizeof(double) * (size_t)(p->nz + 2 * NG));
    h->p.z = h->zh;
  }
  h->L = make_layout(p->nx, p->ny, p->nz);
  h->st = (cudaStream_t)stream;
  h->esz = p->precision == 64 ? 8 : 4;
  h->ws = (char*)workspace;
  h->ws_bytes = ws_bytes;
  h->f[0] = h->ws + o.f0;
  h->f[1] = h->ws + o.f1;
  h->df = h->ws + o.df;
  h->lnrho0 = h->ws + o.lnrho0;
  h->wtab = h->ws + o.wtab;
  h->wptab = h->ws + o.wptab;
  h->bz = h->ws + o.bz;
  h->axt = h->ws + o.axt;
  h->ayt = h->ws + o.ayt;
  h->v0 = h->ws + o.v0;
  h->v1 = h->ws + o.v1;
  h->red = (double*)(h->ws + o.red);
  h->cfl = h->red + (size_t)RED_BLOCKS_MAX * 8;
  h->ss = (StepState*)(h->ws + o.ss);
  h->bgtab = h->ws + o.bg;
  h->ztab = h->ws + o.ztab;
  h->zt64 = (double*)(h->ws + o.zt64);
  h->bj = h->ws + o.bj;
  h->sw = h->ws + o.sw;
  h->ksw = swamp_first_layer(p);
  h->abg_mode = p->a_background != 0;
  if (h->abg_mode) {
    h->abB = h->ws + o.abB;
    h->abL = h->ws + o.abL;
    h->abgR = h->ws + o.abgR;
    h->abg0 = (double*)(h->ws + o.abg0);
    h->at64 = (double*)(h->ws + o.at64);
    h->atrel = h->ws + o.atrel;
  }
  if (p->adjoint) {
    h->s2 = h->ws + o.s2;
    h->fbar = h->ws + o.fbar;
    h->dbar = h->ws + o.dbar;
    h->gbar = h->ws + o.gbar;
    h->coef = h->ws + o.coef;
    h->thbar = (double*)(h->ws + o.thbar);
  }
  h->have_fft = p->bc_z == 0;
  {
    const char* v = getenv("MHD_RK_VARIANT");
    h->tiled = p->precision == 32 && !(v && strcmp(v, "simple") == 0);
    h->split = h->tiled && !(v && strcmp(v, "fused") == 0);
    h->pair = h->split && !(v && (strcmp(v, "tiled") == 0 || strcmp(v, "split") == 0)) &&
              rk_pair_supported(h->L);
    if ((h->abg_mode || h->zh) && h->tiled && !h->pair) {
      // the background tables and the vertical grid are read by the pair
      // kernel and the simple kernel only
      free(h->zh);
      free(h);
      return fail(nullptr, MHD_ERR_UNSUPPORTED,
                  "a_background and a non-uniform z grid need the default FP32 kernel (nx even, nx >= 8, ny >= 6) "
                  "or MHD_RK_VARIANT=simple");
    }
    if (h->abg_mode) h->split = false;
    const char* va = getenv("MHD_ADJ_VARIANT");
    h->adj_tiled = !(va && strcmp(va, "simple") == 0);
    h->adj_zm = h->adj_tiled && !(va && strcmp(va, "tiled3d") == 0);
    h->adj_pair = h->adj_zm && h->pair;
  }
  h->t0 = 0.0;
  h->t1 = 0.0;
  h->dbg_skip_plane = INT_MIN;
  snprintf(h->err, sizeof h->err, "no error");

  int rc = MHD_OK;
  // host tables: density ghosts, swamp weights
  {
    size_t es = h->esz;
    std::vector<char> buf(8 * es + 2 * (size_t)p->nz * es);
    for (int m = 0; m < NG; ++m) {
      double v = lnrho0[m];  // z index m - 3
      if (es == 8) ((double*)buf.data())[m] = v; else ((float*)buf.data())[m] = (float)v;
    }
    rc = cuda_check(h, cudaMemcpy(h->lnrho0, buf.data(), 8 * es, cudaMemcpyHostToDevice), "upload lnrho0");
    std::vector<double> w(p->nz), wp(p->nz);
    for (int k = 0; k < p->nz; ++k) swamp_weight(p, zpos(p, k), &w[k], &wp[k]);
    char* wb = buf.data() + 8 * es;
    for (int k = 0; k < p->nz; ++k) {
      if (es == 8) { ((double*)wb)[k] = w[k]; ((double*)wb)[p->nz + k] = wp[k]; }
      else { ((float*)wb)[k] = (float)w[k]; ((float*)wb)[p->nz + k] = (float)wp[k]; }
    }
    if (!rc) rc = cuda_check(h, cudaMemcpy(h->wtab, wb, (size_t)p->nz * es, cudaMemcpyHostToDevice), "upload w");
    if (!rc) rc = cuda_check(h, cudaMemcpy(h->wptab, wb + (size_t)p->nz * es, (size_t)p->nz * es,
                                            cudaMemcpyHostToDevice), "upload wp");
  }
  if (!rc && h->have_fft) rc = upload_fft_tables(h, o);
  if (!rc && h->have_fft) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    rc = cuda_check(h, cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi), "side stream");
    if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->evf, cudaEventDisableTiming), "fork event");
    if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->evj, cudaEventDisableTiming), "join event");
    for (int i = 0; i < 2 && !rc; ++i) {
      rc = cuda_check(h, cudaStreamCreateWithPriority(&h->ps.s[i], cudaStreamNonBlocking, hi), "plane stream");
      if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ps.join[i], cudaEventDisableTiming), "plane event");
    }
    if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ps.fork, cudaEventDisableTiming), "plane event");
  }
  if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->evc, cudaEventDisableTiming), "copy event");
  if (!rc && h->tiled) {
    for (int s = 0; s < 2 && !rc; ++s)
      if (make_state_tensor_map(&h->tm[s], h->L, h->f[s]) != 0)
        rc = fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for state set %d", s);
    if (!rc && p->adjoint && make_state_tensor_map(&h->tm[2], h->L, h->s2) != 0)
      rc = fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for the adjoint substep state");
    for (int s = 0; s < 2 && !rc; ++s)
      if (make_state_tensor_map(&h->tma[s], h->L, h->f[s], 3) != 0 ||
          make_state_tensor_map(&h->tmr[s], h->L, h->f[s], 5) != 0)
        rc = fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for the split boxes of state set %d", s);
    if (!rc && make_state_tensor_map(&h->tmdf, h->L, h->df, NF, 32, 8) != 0)
      rc = fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for the RK accumulator");
    if (!rc && p->adjoint && make_state_tensor_map(&h->tmdbar, h->L, h->dbar, NF, 32, 8) != 0)
      rc = fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for the adjoint accumulator");
  }
  if (!rc) {
    StepState s0;
    memset(&s0, 0, sizeof s0);
    rc = cuda_check(h, cudaMemcpy(h->ss, &s0, sizeof s0, cudaMemcpyHostToDevice), "init step state");
  }
  if (!rc) {
    // zero the driver (no nudging target until mhd_set_driver)
    rc = cuda_check(h, cudaMemsetAsync(h->bz, 0, (size_t)(o.red - o.bz), h->st), "zero driver");
  }
  if (!rc && h->abg_mode) {
    // no background until mhd_set_a_background: every table zero
    rc = cuda_check(h, cudaMemsetAsync(h->ws + o.abB, 0, o.at64 - o.abB, h->st), "zero background tables");
    if (!rc) rc = cuda_check(h, cudaMemsetAsync(h->atrel, 0, 2 * (size_t)p->nx * p->ny * h->esz, h->st),
                             "zero background target");
  }
  // background profiles: ln T from the given profile or the layer means of
  // the initial state (staged in the accumulator buffer)
  if (!rc) {
    std::vector<double> tmean((size_t)p->nz, 0.0);
    if (!lnT0 && p->bc_z == 0) {
      size_t bytes = (size_t)NF * p->nx * p->ny * p->nz * h->esz;
      rc = cuda_check(h, cudaMemcpyAsync(h->df, init_state, bytes, kind_in(mem), h->st), "stage state");
      if (!rc) {
        if (h->esz == 8) launch_layer_mean<double>(h->L, (const double*)h->df, LT, h->red, h->st);
        else launch_layer_mean<float>(h->L, (const float*)h->df, LT, h->red, h->st);
        rc = cuda_check(h, cudaMemcpyAsync(tmean.data(), h->red, (size_t)p->nz * 8, cudaMemcpyDeviceToHost, h->st),
                        "layer means");
      }
      if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "layer means synchronize");
    }
    if (!rc) rc = h->esz == 8 ? upload_background<double>(h, lnrho0, lnT0, tmean.data())
                              : upload_background<float>(h, lnrho0, lnT0, tmean.data());
  }
  if (!rc) rc = mhd_write(h, init_state, mem);
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "create synchronize");
  if (rc) {
    snprintf(g_err, sizeof g_err, "%s", h->err);
    release_side(h);
    free(h->zh);
    free(h);
    return rc;
  }
  *out = h;
  return MHD_OK;
}

extern "C" int mhd_write(mhd_handle h, const void* src, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!src) return fail(h, MHD_ERR_ARG, "src is NULL");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  const Layout& L = h->L;
  size_t bytes = (size_t)NF * L.nx * L.ny * L.nz * h->esz;
  int rc = cuda_check(h, cudaMemcpyAsync(h->df, src, bytes, kind_in(mem), h->st), "copy state in");
  if (rc) return rc;
  // a state written afresh may be stepped again: clear the halt flag
  rc = cuda_check(h, cudaMemsetAsync(&h->ss->nonfinite, 0, sizeof(int), h->st), "clear status");
  if (rc) return rc;
  for (int s = 0; s < 2; ++s) {
    if (h->esz == 8) {
      double* f = (double*)h->f[s];
      cudaMemsetAsync(f, 0, (size_t)NF * L.fs * 8, h->st);
      launch_unpack<double>(L, h->bgd, (const double*)h->df, f, h->st);
      launch_rims<double>(L, f, 0, L.nz, h->st);
      if (h->p.bc_z == 0) launch_init_u_ghosts<double>(L, f, h->st);
    } else {
      float* f = (float*)h->f[s];
      cudaMemsetAsync(f, 0, (size_t)NF * L.fs * 4, h->st);
      launch_unpack<float>(L, h->bgf, (const float*)h->df, f, h->st);
      launch_rims<float>(L, f, 0, L.nz, h->st);
      if (h->p.bc_z == 0) launch_init_u_ghosts<float>(L, f, h->st);
    }
  }
  h->cur = 0;
  rc = cuda_check(h, cudaSuccess, "state unpack");
  if (rc) return rc;
  if (mem == MHD_MEM_HOST) rc = cuda_check(h, cudaStreamSynchronize(h->st), "write synchronize");
  return rc;
}

// A stored about a background: the nudging target relative to the
// background's photospheric layer, A_target - A_bg(k = 0), with A_target
// inverted again in FP64 (the stored axt, ayt are rounded to the state
// precision, which at |A| ~ 1e2 would put FP32 rounding noise into the
// nudging at the photosphere).
static int background_target(mhd_ctx* h) {
  const long long n2 = (long long)h->p.nx * h->p.ny;
  double* bz64 = h->at64 + 2 * n2;
  if (h->esz == 8) launch_widen<double>((const double*)h->bz, bz64, n2, h->st);
  else launch_widen<float>((const float*)h->bz, bz64, n2, h->st);
  launch_atarget<double>(h->fp, bz64, h->at64, h->at64 + n2, h->st);
  if (h->esz == 8) launch_abg_target<double>(h->at64, h->abg0, (double*)h->atrel, 2 * n2, h->st);
  else launch_abg_target<float>(h->at64, h->abg0, (float*)h->atrel, 2 * n2, h->st);
  return cuda_check(h, cudaSuccess, "background nudging target");
}

template <typename R>
static void background_tables(mhd_ctx* h, const double* a64) {
  const Layout& L = h->L;
  launch_abg_tables<R>(L, h->p.dx, h->p.dy, h->p.dz, h->p.z ? h->zt64 : nullptr, a64, (R*)h->abB,
                       (R*)h->abB + 3LL * L.nx * L.ny * L.nz,
                       (R*)h->abL, h->ksw, h->abg0, (R*)h->abgR, h->st);
}

extern "C" int mhd_set_a_background(mhd_handle h, const double* a_bg, const void* a_pert, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!h->abg_mode) return fail(h, MHD_ERR_ARG, "the handle was created with a_background = 0");
  if (!a_bg) return fail(h, MHD_ERR_ARG, "a_bg is NULL");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  const Layout& L = h->L;
  const size_t n3 = (size_t)L.nx * L.ny * L.nz;
  // FP64 background, ghost-filled, in the RK accumulator's memory (fields
  // 0..2 of an FP64 state layout: 24 fs bytes of the accumulator's 8 fs esz);
  // a host input is staged in the other state set first
  double* a64 = (double*)h->df;
  const double* src = a_bg;
  int rc = MHD_OK;
  if (mem == MHD_MEM_HOST) {
    double* stage = (double*)h->f[1 - h->cur];
    rc = cuda_check(h, cudaMemcpyAsync(stage, a_bg, 3 * n3 * 8, cudaMemcpyHostToDevice, h->st), "copy background in");
    src = stage;
  }
  if (!rc) rc = cuda_check(h, cudaMemsetAsync(a64, 0, (size_t)3 * L.fs * 8, h->st), "zero background scratch");
  if (rc) return rc;
  launch_abg_unpack64(L, src, a64, h->st);
  if (h->have_fft) launch_pfe<double>(h->fp, L, a64, h->ss, h->st, nullptr);
  else launch_abg_zper(L, a64, h->st);
  if (h->esz == 8) background_tables<double>(h, a64);
  else background_tables<float>(h, a64);
  rc = cuda_check(h, cudaSuccess, "background tables");
  if (rc) return rc;
  // the state's A is now the perturbation: a_pert, or zero
  const size_t abytes = (size_t)3 * L.fs * h->esz;
  rc = cuda_check(h, cudaMemsetAsync(h->f[h->cur], 0, abytes, h->st), "zero A");
  if (!rc && a_pert) {
    const void* ps = a_pert;
    if (mem == MHD_MEM_HOST) {
      rc = cuda_check(h, cudaMemcpyAsync(h->df, a_pert, 3 * n3 * h->esz, cudaMemcpyHostToDevice, h->st),
                      "copy perturbation in");
      ps = h->df;
    }
    if (!rc) {
      if (h->esz == 8) launch_abg_pert<double>(L, (const double*)ps, (double*)h->f[h->cur], h->st);
      else launch_abg_pert<float>(L, (const float*)ps, (float*)h->f[h->cur], h->st);
      rc = cuda_check(h, cudaSuccess, "perturbation");
    }
  }
  if (!rc && h->have_fft && h->driver_set) rc = background_target(h);
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "background synchronize");
  return rc;
}

extern "C" int mhd_fma_peak(int precision, void* scratch, void* stream, double* flops_per_s) {
  if ((precision != 32 && precision != 64) || !scratch || !flops_per_s) {
    set_global_error("mhd_fma_peak: precision 32 or 64, a device scratch pointer and an output are required");
    return MHD_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = 8 * (sms > 0 ? sms : 1);        // 8 blocks of 256 threads per SM
  const int iters = precision == 64 ? 1 << 12 : 1 << 16;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 0.f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    cudaEventRecord(a, st);
    if (precision == 64) launch_fma_probe<double>((double*)scratch, grid, iters, st);
    else launch_fma_probe<float>((float*)scratch, grid, iters, st);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !(best > 0.f)) {
    set_global_error("mhd_fma_peak: %s", cudaGetErrorString(e));
    return MHD_ERR_CUDA;
  }
  *flops_per_s = 2.0 * 8.0 * (double)iters * 256.0 * (double)grid / (best * 1e-3);
  return MHD_OK;
}

extern "C" int mhd_debug_skip_copy(mhd_handle h, int plane, int wait_limit) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!(h->esz == 4 && h->pair)) return fail(h, MHD_ERR_UNSUPPORTED, "the hook acts on the FP32 pair kernel only");
  if (plane < -NG || plane > h->p.nz + NG - 1) return fail(h, MHD_ERR_ARG, "plane must be in -3 .. nz + 2");
  if (wait_limit < 1) return fail(h, MHD_ERR_ARG, "wait_limit must be >= 1");
  h->dbg_skip_plane = plane;
  h->dbg_wait_limit = wait_limit;
  return MHD_OK;
}

extern "C" int mhd_set_driver(mhd_handle h, const void* bz, const void* v0, const void* v1, double t0,
                              double t1, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!bz || !v0 || !v1) return fail(h, MHD_ERR_ARG, "bz, v0, v1 are required");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  if (!(t1 > t0)) return fail(h, MHD_ERR_ARG, "driver times need t1 > t0");
  size_t n2 = (size_t)h->p.nx * h->p.ny * h->esz;
  int rc = cuda_check(h, cudaMemcpyAsync(h->bz, bz, n2, kind_in(mem), h->st), "copy bz");
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(h->v0, v0, 2 * n2, kind_in(mem), h->st), "copy v0");
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(h->v1, v1, 2 * n2, kind_in(mem), h->st), "copy v1");
  if (!rc) rc = cuda_check(h, cudaEventRecord(h->evc, h->st), "copy event");
  if (rc) return rc;
  h->t0 = t0;
  h->t1 = t1;
  if (h->have_fft) {
    if (h->esz == 8) launch_atarget<double>(h->fp, (const double*)h->bz, (double*)h->axt, (double*)h->ayt, h->st);
    else launch_atarget<float>(h->fp, (const float*)h->bz, (float*)h->axt, (float*)h->ayt, h->st);
    rc = cuda_check(h, cudaSuccess, "magnetogram inversion");
    if (rc) return rc;
    if (h->abg_mode) rc = background_target(h);
    if (rc) return rc;
  }
  h->driver_set = true;
  // host buffers may be reused once the copies are done; the inversion
  // runs on behind the return
  if (mem == MHD_MEM_HOST) rc = cuda_check(h, cudaEventSynchronize(h->evc), "driver copies");
  return rc;
}

extern "C" int mhd_step(mhd_handle h, int nsteps) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (nsteps < 0) return fail(h, MHD_ERR_ARG, "nsteps < 0");
  for (int n = 0; n < nsteps; ++n) {
    bool stats = h->p.stats_every > 0 && (h->host_steps % h->p.stats_every) == 0;
    if (h->esz == 8) run_step<double>(h, stats); else run_step<float>(h, stats);
    h->host_steps++;
  }
  return cuda_check(h, cudaSuccess, "step launch");
}

extern "C" int mhd_read(mhd_handle h, int field, void* dst, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!dst) return fail(h, MHD_ERR_ARG, "dst is NULL");
  if (field < -1 || field >= NF) return fail(h, MHD_ERR_ARG, "field must be -1..7");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  const Layout& L = h->L;
  size_t bytes = (size_t)(field < 0 ? NF : 1) * L.nx * L.ny * L.nz * h->esz;
  void* tgt = mem == MHD_MEM_HOST ? h->df : dst;
  if (h->esz == 8) launch_pack<double>(L, h->bgd, (const double*)h->f[h->cur], (double*)tgt, field, h->st);
  else launch_pack<float>(L, h->bgf, (const float*)h->f[h->cur], (float*)tgt, field, h->st);
  int rc = cuda_check(h, cudaSuccess, "pack");
  if (rc) return rc;
  if (mem == MHD_MEM_HOST) {
    rc = cuda_check(h, cudaMemcpyAsync(dst, h->df, bytes, cudaMemcpyDeviceToHost, h->st), "copy out");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "read synchronize");
  }
  return rc;
}

extern "C" int mhd_read_plane(mhd_handle h, int field, int k, void* dst, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!dst) return fail(h, MHD_ERR_ARG, "dst is NULL");
  if (field < 0 || field >= NF) return fail(h, MHD_ERR_ARG, "field must be 0..7");
  if (k < 0 || k >= h->L.nz) return fail(h, MHD_ERR_ARG, "k must be 0..nz-1");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  const Layout& L = h->L;
  void* tgt = mem == MHD_MEM_HOST ? h->df : dst;
  if (h->esz == 8) launch_pack_plane<double>(L, h->bgd, (const double*)h->f[h->cur], (double*)tgt, field, k, h->st);
  else launch_pack_plane<float>(L, h->bgf, (const float*)h->f[h->cur], (float*)tgt, field, k, h->st);
  int rc = cuda_check(h, cudaSuccess, "pack plane");
  if (rc) return rc;
  if (mem == MHD_MEM_HOST) {
    rc = cuda_check(h, cudaMemcpyAsync(dst, h->df, (size_t)L.nx * L.ny * h->esz, cudaMemcpyDeviceToHost, h->st),
                    "copy plane out");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "read synchronize");
  }
  return rc;
}

extern "C" int mhd_read_padded(mhd_handle h, int which, void* dst, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!dst || (which != 0 && which != 1)) return fail(h, MHD_ERR_ARG, "bad dst or which");
  if (mem != MHD_MEM_DEVICE && mem != MHD_MEM_HOST) return fail(h, MHD_ERR_ARG, "bad mem flag");
  const Layout& L = h->L;
  size_t w = (size_t)(L.nx + 2 * NG) * h->esz;
  size_t rows = (size_t)L.mz * L.my;
  if (which == 0) {
    // state: background added, staged in the accumulator buffer
    if (h->esz == 8) launch_pack_padded<double>(L, h->bgd, (const double*)h->f[h->cur], (double*)h->df, h->st);
    else launch_pack_padded<float>(L, h->bgf, (const float*)h->f[h->cur], (float*)h->df, h->st);
    int rc = cuda_check(h, cudaMemcpyAsync(dst, h->df, (size_t)NF * rows * w, kind_out(mem), h->st), "copy padded");
    if (rc) return rc;
  } else {
    const char* src = (const char*)h->df;
    for (int fl = 0; fl < NF; ++fl) {
      const char* s = src + ((size_t)fl * L.fs + (XOFF - NG)) * h->esz;
      char* d = (char*)dst + (size_t)fl * rows * w;
      int rc = cuda_check(h, cudaMemcpy2DAsync(d, w, s, (size_t)L.mx * h->esz, w, rows, kind_out(mem), h->st),
                          "copy padded");
      if (rc) return rc;
    }
  }
  if (mem == MHD_MEM_HOST) return cuda_check(h, cudaStreamSynchronize(h->st), "read synchronize");
  return MHD_OK;
}

extern "C" int mhd_write_snapshot(mhd_handle h, const char* var_path, const char* grid_path) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!var_path && !grid_path) return fail(h, MHD_ERR_ARG, "no file path given");
  double t, dt;
  int rc = mhd_get_time(h, &t, &dt);  // synchronises; reports a halted handle
  if (rc) return rc;
  const Layout& L = h->L;
  const size_t bytes = (size_t)L.mz * L.my * (L.nx + 2 * NG) * h->esz;
  if (var_path) {
    // outer ghosts consistent with the state, then the padded state with its
    // backgrounds added, staged in the accumulator buffer (free between steps)
    rc = mhd_fill_ghosts(h);
    if (rc) return rc;
    if (h->esz == 8) launch_pack_padded<double>(L, h->bgd, (const double*)h->f[h->cur], (double*)h->df, h->st);
    else launch_pack_padded<float>(L, h->bgf, (const float*)h->f[h->cur], (float*)h->df, h->st);
    rc = cuda_check(h, cudaStreamSynchronize(h->st), "stage padded state");
    if (rc) return rc;
  }
  std::vector<char> host(var_path ? bytes : 0);
  cudaError_t ce = cudaSuccess;
  auto field = [&](int f, FILE* fp) -> bool {
    ce = cudaMemcpyAsync(host.data(), (const char*)h->df + (size_t)f * bytes, bytes, cudaMemcpyDeviceToHost, h->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
    return ce == cudaSuccess && std::fwrite(host.data(), 1, bytes, fp) == bytes;
  };
  const int w = h5_write_snapshot(var_path, grid_path, &h->p, t, field);
  if (ce != cudaSuccess) return cuda_check(h, ce, "copy snapshot field");
  if (w) return fail(h, MHD_ERR_IO, "cannot write the snapshot files (%s, %s)", var_path ? var_path : "-",
                     grid_path ? grid_path : "-");
  return MHD_OK;
}

extern "C" int mhd_h5_write(const char* var_path, const char* grid_path, const mhd_params* p, double t,
                            const void* padded) {
  if (!p) return fail(nullptr, MHD_ERR_ARG, "NULL params");
  const char* bad = check_params(p);
  if (bad) return fail(nullptr, MHD_ERR_ARG, "%s", bad);
  if (!var_path && !grid_path) return fail(nullptr, MHD_ERR_ARG, "no file path given");
  if (var_path && !padded) return fail(nullptr, MHD_ERR_ARG, "NULL state");
  const size_t bytes = (size_t)(p->nz + 2 * NG) * (p->ny + 2 * NG) * (p->nx + 2 * NG) * (p->precision == 64 ? 8 : 4);
  auto field = [&](int f, FILE* fp) -> bool {
    return std::fwrite((const char*)padded + (size_t)f * bytes, 1, bytes, fp) == bytes;
  };
  if (h5_write_snapshot(var_path, grid_path, p, t, field))
    return fail(nullptr, MHD_ERR_IO, "cannot write the snapshot files (%s, %s)", var_path ? var_path : "-",
                grid_path ? grid_path : "-");
  return MHD_OK;
}

extern "C" int mhd_fill_ghosts(mhd_handle h) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (h->esz == 8) ghost_fill<double>(h, (double*)h->f[h->cur]);
  else ghost_fill<float>(h, (float*)h->f[h->cur]);
  return cuda_check(h, cudaSuccess, "ghost fill");
}

extern "C" int mhd_eval_rhs(mhd_handle h, double t, void* dst, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  double r, s;
  driver_weights(h, t, &r, &s);
  double rs[2] = {r, s};
  int rc = cuda_check(h, cudaMemcpyAsync(&h->ss->eval_r, rs, sizeof rs, cudaMemcpyHostToDevice, h->st),
                      "eval weights");
  if (rc) return rc;
  rc = cuda_check(h, cudaMemsetAsync(h->df, 0, (size_t)NF * h->L.fs * h->esz, h->st), "zero df");
  if (rc) return rc;
  if (h->esz == 8) launch_rk_any<double>(h, (const double*)h->f[h->cur], nullptr, -1);
  else launch_rk_any<float>(h, (const float*)h->f[h->cur], nullptr, -1);
  rc = cuda_check(h, cudaSuccess, "rhs");
  if (rc) return rc;
  if (mem == MHD_MEM_HOST) {
    rc = cuda_check(h, cudaStreamSynchronize(h->st), "rhs synchronize");
    if (rc) return rc;
  }
  return mhd_read_padded(h, 1, dst, mem);
}

extern "C" int mhd_compute_dt(mhd_handle h, double* dt) {
  if (!h || !dt) return fail(h, MHD_ERR_ARG, "NULL argument");
  int nb;
  if (h->esz == 8) {
    Phys<double> ph = make_phys<double>(&h->p);
    nb = launch_cfl_partial<double>(h->L, ph, h->bgd, (const double*)h->f[h->cur], (const double*)h->wtab, h->cfl,
                                    h->ss, CflPlanes::all, true, h->st);
  } else {
    Phys<float> ph = make_phys<float>(&h->p);
    nb = launch_cfl_partial<float>(h->L, ph, h->bgf, (const float*)h->f[h->cur], (const float*)h->wtab, h->cfl,
                                   h->ss, CflPlanes::all, true, h->st);
  }
  launch_cfl_finalize(h->cfl, nb, h->ss, h->p.c_adv, h->p.c_diff, 0.0, inv2sum(&h->p), h->t0, h->t1,
                      h->p.t_ramp, 1, h->st);
  int rc = sync_status(h);
  if (rc) return rc;
  return cuda_check(h, cudaMemcpy(dt, &h->ss->probe_dt, sizeof(double), cudaMemcpyDeviceToHost), "read dt");
}

static int fetch_stats(mhd_ctx* h, mhd_stats* out) {
  StepState s;
  int rc = cuda_check(h, cudaMemcpy(&s, h->ss, sizeof s, cudaMemcpyDeviceToHost), "read stats");
  if (rc) return rc;
  memset(out, 0, sizeof *out);
  out->t = s.t;
  out->dt = s.dt;
  out->e_kin = s.stats[0];
  out->e_mag = s.stats[1];
  out->e_th = s.stats[2];
  out->mass = s.stats[3];
  out->flux_net = s.stats[4];
  out->flux_abs = s.stats[5];
  out->divb_max = s.stats[6];
  out->step = s.step;
  out->nonfinite = s.nonfinite;
  return MHD_OK;
}

extern "C" int mhd_compute_stats(mhd_handle h, mhd_stats* out) {
  if (!h || !out) return fail(h, MHD_ERR_ARG, "NULL argument");
  if (h->esz == 8) run_stats<double>(h, (double*)h->f[h->cur]);
  else run_stats<float>(h, (float*)h->f[h->cur]);
  int rc = cuda_check(h, cudaStreamSynchronize(h->st), "stats synchronize");
  if (rc) return rc;
  rc = fetch_stats(h, out);
  if (rc) return rc;
  if (out->nonfinite & 2) return fail(h, MHD_ERR_TIMEOUT, "a device wait exceeded its bound");
  if (out->nonfinite) return fail(h, MHD_ERR_NONFINITE, "non-finite value in the state");
  return MHD_OK;
}

extern "C" int mhd_read_stats(mhd_handle h, mhd_stats* out) {
  if (!h || !out) return fail(h, MHD_ERR_ARG, "NULL argument");
  int rc = cuda_check(h, cudaStreamSynchronize(h->st), "stats synchronize");
  if (rc) return rc;
  rc = fetch_stats(h, out);
  if (rc) return rc;
  if (out->nonfinite & 2) return fail(h, MHD_ERR_TIMEOUT, "a device wait exceeded its bound (time stepping halted)");
  if (out->nonfinite) return fail(h, MHD_ERR_NONFINITE, "non-finite value in the state (time stepping halted)");
  return MHD_OK;
}

extern "C" int mhd_set_time(mhd_handle h, double t) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  double tt = t;
  int rc = cuda_check(h, cudaMemcpyAsync(&h->ss->t, &tt, sizeof(double), cudaMemcpyHostToDevice, h->st), "set time");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "set time synchronize");
  return rc;
}

extern "C" int mhd_get_time(mhd_handle h, double* t, double* dt) {
  if (!h || !t || !dt) return fail(h, MHD_ERR_ARG, "NULL argument");
  double td[2];
  int nf = 0;
  int rc = cuda_check(h, cudaStreamSynchronize(h->st), "time synchronize");
  if (!rc) rc = cuda_check(h, cudaMemcpy(td, &h->ss->t, sizeof td, cudaMemcpyDeviceToHost), "read time");
  if (!rc) rc = cuda_check(h, cudaMemcpy(&nf, &h->ss->nonfinite, sizeof nf, cudaMemcpyDeviceToHost), "read status");
  if (rc) return rc;
  *t = td[0];
  *dt = td[1];
  if (nf & 2) return fail(h, MHD_ERR_TIMEOUT, "a device wait exceeded its bound (time stepping halted)");
  if (nf) return fail(h, MHD_ERR_NONFINITE, "non-finite value in the state (time stepping halted)");
  return MHD_OK;
}

extern "C" int mhd_read_target(mhd_handle h, void* dst, int mem) {
  if (!h || !dst) return fail(h, MHD_ERR_ARG, "NULL argument");
  size_t n2 = (size_t)h->p.nx * h->p.ny * h->esz;
  int rc = cuda_check(h, cudaMemcpyAsync(dst, h->axt, n2, kind_out(mem), h->st), "copy axt");
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync((char*)dst + n2, h->ayt, n2, kind_out(mem), h->st), "copy ayt");
  if (!rc && mem == MHD_MEM_HOST) rc = cuda_check(h, cudaStreamSynchronize(h->st), "target synchronize");
  return rc;
}

// ---- adjoint -----------------------------------------------------------------
extern "C" size_t mhd_checkpoint_bytes(mhd_handle h) {
  return h ? (size_t)NF * h->L.fs * h->esz : 0;
}

extern "C" int mhd_save(mhd_handle h, void* dst, double* t) {
  if (!h || !dst || !t) return fail(h, MHD_ERR_ARG, "NULL argument");
  int rc = cuda_check(h, cudaMemcpyAsync(dst, h->f[h->cur], mhd_checkpoint_bytes(h), cudaMemcpyDeviceToDevice, h->st),
                      "save");
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(t, &h->ss->t, sizeof(double), cudaMemcpyDeviceToHost, h->st), "save t");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "save synchronize");
  return rc;
}

extern "C" int mhd_restore(mhd_handle h, const void* src, double t) {
  if (!h || !src) return fail(h, MHD_ERR_ARG, "NULL argument");
  int rc = cuda_check(h, cudaMemcpyAsync(h->f[h->cur], src, mhd_checkpoint_bytes(h), cudaMemcpyDeviceToDevice, h->st),
                      "restore");
  double tt = t;
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(&h->ss->t, &tt, sizeof(double), cudaMemcpyHostToDevice, h->st),
                           "restore t");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "restore synchronize");
  return rc;
}

static int adjoint_ready(mhd_ctx* h) {
  if (!h->p.adjoint) return fail(h, MHD_ERR_ARG, "handle created without params.adjoint");
  if (h->p.bc_z != 0) return fail(h, MHD_ERR_UNSUPPORTED, "the adjoint is built for bc_z = 0");
  if (!(h->p.dt_fixed > 0.0)) return fail(h, MHD_ERR_ARG, "the adjoint needs a frozen time step (dt_fixed > 0)");
  return MHD_OK;
}

extern "C" int mhd_adjoint_init(mhd_handle h, const void* lam, int mem) {
  if (!h || !lam) return fail(h, MHD_ERR_ARG, "NULL argument");
  int rc = adjoint_ready(h);
  if (rc) return rc;
  const size_t set = (size_t)NF * h->L.fs * h->esz;
  const size_t n2 = (size_t)h->p.nx * h->p.ny;
  rc = cuda_check(h, cudaMemsetAsync(h->fbar, 0, set, h->st), "zero fbar");
  if (!rc) rc = cuda_check(h, cudaMemsetAsync(h->dbar, 0, set, h->st), "zero dbar");
  if (!rc) rc = cuda_check(h, cudaMemsetAsync(h->thbar, 0, 6 * n2 * sizeof(double), h->st), "zero thbar");
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(h->gbar, lam, (size_t)NF * h->p.nx * h->p.ny * h->p.nz * h->esz,
                                              kind_in(mem), h->st), "copy lam");
  if (rc) return rc;
  if (h->esz == 8) {
    launch_adj_unpack<double>(h->L, (const double*)h->gbar, (double*)h->fbar, h->st);
    launch_adj_update<double>(h->L, (double*)h->fbar, (double*)h->dbar, nullptr, 0.0, rk_beta(2), 0, 0, 0, h->ss,
                              h->st);
  } else {
    launch_adj_unpack<float>(h->L, (const float*)h->gbar, (float*)h->fbar, h->st);
    launch_adj_update<float>(h->L, (float*)h->fbar, (float*)h->dbar, nullptr, 0.0, rk_beta(2), 0, 0, 0, h->ss,
                             h->st);
  }
  h->nlaunch += 2;
  rc = cuda_check(h, cudaSuccess, "adjoint init");
  if (!rc && mem == MHD_MEM_HOST) rc = cuda_check(h, cudaStreamSynchronize(h->st), "init synchronize");
  return rc;
}

template <typename R>
static void adjoint_reverse(mhd_ctx* h, R* const (&S)[3], const CUtensorMap* const (&tms)[3]);

template <typename R>
static void adjoint_step_impl(mhd_ctx* h) {
  R* S[3] = {(R*)h->f[h->cur], (R*)h->f[1 - h->cur], (R*)h->s2};
  // forward recompute of the substep states (ghost-filled)
  ghost_fill<R>(h, S[0]);
  launch_cfl_finalize(h->cfl, 0, h->ss, h->p.c_adv, h->p.c_diff, h->p.dt_fixed, inv2sum(&h->p), h->t0, h->t1,
                      h->p.t_ramp, 0, h->st);
  launch_rk_any<R>(h, S[0], S[1], 0);
  ghost_fill<R>(h, S[1]);
  launch_rk_any<R>(h, S[1], S[2], 1);
  ghost_fill<R>(h, S[2]);
  h->nlaunch += 3;  // cfl finalize and the two RK substeps (ghost_fill counts its own)
  const CUtensorMap* tms[3] = {&h->tm[h->cur], &h->tm[1 - h->cur], &h->tm[2]};
  adjoint_reverse<R>(h, S, tms);
}

// The reverse substeps of one step from its three ghost-filled substep
// states S (and, for the FP32 z-march point kernel, their tensor maps).
template <typename R>
static void adjoint_reverse(mhd_ctx* h, R* const (&S)[3], const CUtensorMap* const (&tms)[3]) {
  Phys<R> ph = make_phys<R>(&h->p);
  const Background<R>& bg = bgr<R>(h);
  // reverse substeps
  FFTPlan fpa = h->fp;
  fpa.P = h->fp.Q;   // 9 packed ghost-adjoint planes
  fpa.Q = h->fp.P;   // 3 summed planes
  // tiled gather: it applies the update itself on the layers no ghost rule
  // feeds back into (the ghost-rule transposes touch k < 4 and k >= nz - 4)
  const bool tg = h->adj_tiled && adj_gather_tiled_ok(h->L);
  int klo = 0, khi = 0;
  if (tg && h->p.nz - NG - 1 > NG + 1) {
    klo = NG + 1;
    khi = h->p.nz - NG - 1;
  }
  // Between reverse steps D already holds beta_2 F, the first update of the
  // next step: alpha_0 = 0 makes the accumulator's own adjoint vanish at a
  // step boundary, so the last substep leaves D = beta_2 F (and
  // mhd_adjoint_init starts from D = beta_2 lam).
  for (int s = 2; s >= 0; --s) {
    const double alpha = rk_alpha(s), beta = rk_beta(s > 0 ? s - 1 : 2);
    if (sizeof(R) == 4 && h->adj_pair)
      launch_adj_point_pair(tms[s], &h->tmdbar, h->L, *(const Phys<float>*)&ph, h->bgf, (const float*)h->dbar,
                            (float*)h->coef, h->thbar, (const float*)h->wtab, (const float*)h->wptab, h->ss, s,
                            h->p.dx, h->p.dy, h->p.dz, h->st);
    else if (sizeof(R) == 4 && h->tiled && h->adj_tiled)
      launch_adj_point_tiled(tms[s], h->L, *(const Phys<float>*)&ph, h->bgf, (const float*)h->dbar,
                             (float*)h->coef, h->thbar, (const float*)h->wtab, (const float*)h->wptab, h->ss, s,
                             h->p.dx, h->p.dy, h->p.dz, h->st);
    else
      launch_adj_point<R>(h->L, ph, bg, S[s], (const R*)h->dbar, (R*)h->coef, h->thbar, (const R*)h->wtab,
                          (const R*)h->wptab, h->ss, s, h->st);
    if (tg && h->adj_zm)
      launch_adj_gather_zm<R>(h->L, ph, (const R*)h->coef, (R*)h->dbar, (R*)h->gbar, (R*)h->fbar, alpha, beta, klo,
                              khi, h->ss, h->st);
    else if (tg)
      launch_adj_gather_tiled<R>(h->L, ph, (R*)h->coef, (R*)h->dbar, (R*)h->gbar, (R*)h->fbar, alpha, beta, klo, khi,
                                 h->ss, h->st);
    else
      launch_adj_gather<R>(h->L, ph, (const R*)h->coef, (const R*)h->dbar, (R*)h->gbar, h->ss, h->st);
    launch_adj_bc<R>(h->L, ph, bg, S[s], (R*)h->gbar, (R)h->p.dz, h->ss, h->st);
    launch_pfe_adjoint<R>(fpa, h->L, (R*)h->gbar, h->ss, h->st);
    launch_adj_update<R>(h->L, (R*)h->fbar, (R*)h->dbar, (const R*)h->gbar, alpha, beta, 1, klo, khi, h->ss, h->st);
    h->nlaunch += (tg && !h->adj_zm) ? 8 : 7;  // point, [fold], gather, bc, 3 FFT, update
  }
}

extern "C" int mhd_adjoint_step(mhd_handle h) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  int rc = adjoint_ready(h);
  if (rc) return rc;
  if (h->esz == 8) adjoint_step_impl<double>(h); else adjoint_step_impl<float>(h);
  return cuda_check(h, cudaSuccess, "adjoint step");
}

// ---- tapes: a step's three substep states kept for its adjoint ------------------
// layout: the three state sets, then 256 bytes holding the step's start time
extern "C" size_t mhd_tape_bytes(mhd_handle h) { return h ? 3 * mhd_checkpoint_bytes(h) + 256 : 0; }

static int tape_supported(mhd_ctx* h, const void* tape) {
  if (!tape) return fail(h, MHD_ERR_ARG, "tape is NULL");
  if (((uintptr_t)tape & 255u) != 0) return fail(h, MHD_ERR_ARG, "tape must be 256-byte aligned");
  if (h->esz == 4 && !(h->pair || !h->tiled))
    return fail(h, MHD_ERR_UNSUPPORTED, "tapes need the default FP32 kernel or MHD_RK_VARIANT=simple");
  if (h->esz == 4 && h->p.adjoint && h->tiled && h->adj_tiled && !h->adj_pair)
    return fail(h, MHD_ERR_UNSUPPORTED, "tapes need the default FP32 adjoint kernels");
  return MHD_OK;
}

static int tape_maps(mhd_ctx* h, const void* tape, CUtensorMap* maps) {
  if (h->esz != 4 || !h->tiled) return MHD_OK;  // the one-thread-per-cell kernels take plain pointers
  const size_t set = mhd_checkpoint_bytes(h);
  for (int s = 0; s < 3; ++s)
    if (make_state_tensor_map(&maps[s], h->L, (char*)tape + s * set) != 0)
      return fail(h, MHD_ERR_CUDA, "cuTensorMapEncodeTiled failed for tape state %d", s);
  return MHD_OK;
}

template <typename R>
static void run_step_taped(mhd_ctx* h, char* tape, const CUtensorMap* maps, bool stats) {
  const size_t set = mhd_checkpoint_bytes(h);
  Phys<R> ph = make_phys<R>(&h->p);
  R* S0 = (R*)h->f[h->cur];
  R* T[3] = {(R*)tape, (R*)(tape + set), (R*)(tape + 2 * set)};
  const bool adaptive = !(h->p.dt_fixed > 0.0);
  ghost_fill<R>(h, S0);
  if (stats) run_stats<R>(h, S0);
  {
    ClassTimer ct(h, MHD_KC_CFL, adaptive ? 2 : 1);
    int nb = 0;
    if (adaptive)
      nb = launch_cfl_partial<R>(h->L, ph, bgr<R>(h), S0, (const R*)h->wtab, h->cfl, h->ss, CflPlanes::all, true,
                                 h->st);
    launch_cfl_finalize(h->cfl, nb, h->ss, h->p.c_adv, h->p.c_diff, h->p.dt_fixed, inv2sum(&h->p), h->t0, h->t1,
                        h->p.t_ramp, 0, h->st);
  }
  // the ghost-filled substep inputs go to the tape: S0 by a copy, S1 and S2
  // as the RK kernel's outputs (filled in place there)
  cudaMemcpyAsync(T[0], S0, set, cudaMemcpyDeviceToDevice, h->st);
  {
    ClassTimer ct(h, MHD_KC_RK, 1);
    launch_rk_any<R>(h, S0, T[1], 0);
  }
  ghost_fill<R>(h, T[1]);
  {
    ClassTimer ct(h, MHD_KC_RK, 1);
    launch_rk_any<R>(h, T[1], T[2], 1, maps ? &maps[1] : nullptr);
  }
  ghost_fill<R>(h, T[2]);
  {
    ClassTimer ct(h, MHD_KC_RK, 1);
    launch_rk_any<R>(h, T[2], (R*)h->f[1 - h->cur], 2, maps ? &maps[2] : nullptr);
  }
  h->cur = 1 - h->cur;
}

extern "C" int mhd_step_taped(mhd_handle h, void* tape) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  int rc = tape_supported(h, tape);
  if (rc) return rc;
  alignas(64) CUtensorMap maps[3];
  rc = tape_maps(h, tape, maps);
  if (rc) return rc;
  const bool use_maps = h->esz == 4 && h->tiled;
  // the start time, kept with the states
  rc = cuda_check(h, cudaMemcpyAsync((char*)tape + 3 * mhd_checkpoint_bytes(h), &h->ss->t, sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->st), "tape t");
  if (rc) return rc;
  const bool stats = h->p.stats_every > 0 && (h->host_steps % h->p.stats_every) == 0;
  if (h->esz == 8) run_step_taped<double>(h, (char*)tape, nullptr, stats);
  else run_step_taped<float>(h, (char*)tape, use_maps ? maps : nullptr, stats);
  h->host_steps++;
  return cuda_check(h, cudaSuccess, "taped step");
}

extern "C" int mhd_adjoint_step_taped(mhd_handle h, const void* tape) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  int rc = adjoint_ready(h);
  if (!rc) rc = tape_supported(h, tape);
  if (rc) return rc;
  alignas(64) CUtensorMap maps[3];
  rc = tape_maps(h, tape, maps);
  if (rc) return rc;
  rc = cuda_check(h, cudaMemcpyAsync(&h->ss->t, (const char*)tape + 3 * mhd_checkpoint_bytes(h), sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->st), "tape t");
  if (rc) return rc;
  // the substep times and driver weights of the recorded step
  launch_cfl_finalize(h->cfl, 0, h->ss, h->p.c_adv, h->p.c_diff, h->p.dt_fixed, inv2sum(&h->p), h->t0, h->t1,
                      h->p.t_ramp, 0, h->st);
  h->nlaunch += 1;
  const size_t set = mhd_checkpoint_bytes(h);
  char* tp = (char*)tape;
  const CUtensorMap* tms[3] = {&maps[0], &maps[1], &maps[2]};
  if (h->esz == 8) {
    double* const S[3] = {(double*)tp, (double*)(tp + set), (double*)(tp + 2 * set)};
    adjoint_reverse<double>(h, S, tms);
  } else {
    float* const S[3] = {(float*)tp, (float*)(tp + set), (float*)(tp + 2 * set)};
    adjoint_reverse<float>(h, S, tms);
  }
  return cuda_check(h, cudaSuccess, "taped adjoint step");
}

extern "C" int mhd_adjoint_read(mhd_handle h, void* lam, void* grad_bz, void* grad_v0, void* grad_v1, int mem) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  int rc = adjoint_ready(h);
  if (rc) return rc;
  const size_t n2 = (size_t)h->p.nx * h->p.ny;
  const size_t n3b = (size_t)NF * n2 * h->p.nz * h->esz;
  // results are staged in the coefficient buffer, then copied out
  char* stage = (char*)h->coef;
  if (lam) {
    if (h->esz == 8) launch_adj_pack<double>(h->L, h->p.bc_z, (const double*)h->fbar, (double*)stage, h->st);
    else launch_adj_pack<float>(h->L, h->p.bc_z, (const float*)h->fbar, (float*)stage, h->st);
    rc = cuda_check(h, cudaMemcpyAsync(lam, stage, n3b, kind_out(mem), h->st), "copy lam");
    if (rc) return rc;
  }
  char* stage2 = stage + (n3b + 255) / 256 * 256;
  if (grad_v0 || grad_v1) {
    if (h->esz == 8) launch_d2r<double>(h->thbar + 2 * n2, (double*)stage2, 4 * n2, h->st);
    else launch_d2r<float>(h->thbar + 2 * n2, (float*)stage2, 4 * n2, h->st);
    if (grad_v0) rc = cuda_check(h, cudaMemcpyAsync(grad_v0, stage2, 2 * n2 * h->esz, kind_out(mem), h->st), "v0");
    if (!rc && grad_v1)
      rc = cuda_check(h, cudaMemcpyAsync(grad_v1, stage2 + 2 * n2 * h->esz, 2 * n2 * h->esz, kind_out(mem), h->st),
                      "v1");
    if (rc) return rc;
  }
  if (grad_bz) {
    char* stage3 = stage2 + (4 * n2 * h->esz + 255) / 256 * 256;
    if (h->esz == 8) launch_atarget_adjoint<double>(h->fp, h->thbar, h->thbar + n2, (double*)stage3, h->st);
    else launch_atarget_adjoint<float>(h->fp, h->thbar, h->thbar + n2, (float*)stage3, h->st);
    rc = cuda_check(h, cudaMemcpyAsync(grad_bz, stage3, n2 * h->esz, kind_out(mem), h->st), "bz");
    if (rc) return rc;
  }
  rc = cuda_check(h, cudaSuccess, "adjoint read");
  if (!rc && mem == MHD_MEM_HOST) rc = cuda_check(h, cudaStreamSynchronize(h->st), "read synchronize");
  return rc;
}

extern "C" int mhd_bz_plane(mhd_handle h, const void* state, int k, void* out) {
  if (!h || !state || !out) return fail(h, MHD_ERR_ARG, "NULL argument");
  if (k < 0 || k >= h->p.nz) return fail(h, MHD_ERR_ARG, "layer out of range");
  if (h->esz == 8)
    launch_bz_plane<double>(h->p.nx, h->p.ny, h->p.nz, k, h->p.dx, h->p.dy, (const double*)state, (double*)out, 0,
                            nullptr, nullptr, h->st);
  else
    launch_bz_plane<float>(h->p.nx, h->p.ny, h->p.nz, k, h->p.dx, h->p.dy, (const float*)state, (float*)out, 0,
                           nullptr, nullptr, h->st);
  return cuda_check(h, cudaSuccess, "bz plane");
}

extern "C" int mhd_bz_plane_adjoint(mhd_handle h, const void* bbar, int k, void* lam) {
  if (!h || !bbar || !lam) return fail(h, MHD_ERR_ARG, "NULL argument");
  if (k < 0 || k >= h->p.nz) return fail(h, MHD_ERR_ARG, "layer out of range");
  int rc = cuda_check(h, cudaMemsetAsync(lam, 0, (size_t)NF * h->p.nx * h->p.ny * h->p.nz * h->esz, h->st), "zero lam");
  if (rc) return rc;
  if (h->esz == 8)
    launch_bz_plane<double>(h->p.nx, h->p.ny, h->p.nz, k, h->p.dx, h->p.dy, nullptr, nullptr, 1,
                            (const double*)bbar, (double*)lam, h->st);
  else
    launch_bz_plane<float>(h->p.nx, h->p.ny, h->p.nz, k, h->p.dx, h->p.dy, nullptr, nullptr, 1, (const float*)bbar,
                           (float*)lam, h->st);
  return cuda_check(h, cudaSuccess, "bz plane adjoint");
}

static void drop_events(mhd_ctx* h) {
  if (!h->evs) return;
  for (auto& e : *h->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  h->evs->clear();
}

extern "C" int mhd_profile(mhd_handle h, int enable) {
  if (!h) return fail(nullptr, MHD_ERR_ARG, "NULL handle");
  if (!h->evs) h->evs = new std::vector<mhd_ctx::Ev>();
  if (enable && !h->prof) drop_events(h);
  h->prof = enable != 0;
  h->serial = enable == 2;
  return MHD_OK;
}

extern "C" int mhd_read_profile(mhd_handle h, double* ms, long long* launches) {
  if (!h || !ms || !launches) return fail(h, MHD_ERR_ARG, "NULL argument");
  int rc = cuda_check(h, cudaStreamSynchronize(h->st), "profile synchronize");
  if (rc) return rc;
  for (int c = 0; c < MHD_NKC; ++c) { ms[c] = 0.0; launches[c] = 0; }
  if (h->evs) {
    for (auto& e : *h->evs) {
      float t = 0.f;
      cudaEventElapsedTime(&t, e.a, e.b);
      ms[e.cls] += t;
      launches[e.cls] += e.nk;
    }
    drop_events(h);
  }
  return cuda_check(h, cudaSuccess, "profile read");
}

extern "C" long long mhd_launch_count(mhd_handle h) { return h ? h->nlaunch : 0; }

extern "C" void mhd_destroy(mhd_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  release_side(h);
  drop_events(h);
  delete h->evs;
  free(h->zh);
  free(h);
}

extern "C" const char* mhd_last_error(mhd_handle h) { return h ? h->err : g_err; }
