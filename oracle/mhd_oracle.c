/*
 * mhd_oracle.c -- plain, slow, FP64 CPU oracle of one driven coronal MHD
 * time step (Bourdin 2019, "Driving solar coronal MHD simulations on
 * high-performance computers").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library: every stencil weight, boundary rule and Fourier multiplier is
 * written out here again from the scheme.
 *
 * State: 8 fields (Ax, Ay, Az, ux, uy, uz, ln rho, ln T) -- the variables the
 * paper's snapshots hold (Sect. 5.3, var.h5 content) -- on a padded grid with
 * 3 ghost cells per side (Sect. 2.4 and 2.5 speak of three ghost layers),
 * layout [field][k+3][j+3][i+3], x fastest, i in [-3, nx+3), etc.
 *
 * The paper describes only the additions to the MHD core; the bulk
 * discretisation (sixth-order centred differences, low-storage RK3, CFL rule,
 * ln-variable MHD equations) is the textbook reading written out in the
 * comments below.  Every function follows those equations literally: plain
 * loops, no blocking, no fusion.
 *
 * Parity pins: see tests/test_oracle_*.py.  The whole-run physics of a
 * driven box is "parity unpinned" (the paper prints no numerical solution);
 * each building block is pinned against closed forms and invariants.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG 3
enum { F_AX, F_AY, F_AZ, F_UX, F_UY, F_UZ, F_LNRHO, F_LNTT, NFIELD };

/* parameter vector indices (the Python wrapper fills the same order) */
enum {
  P_DX, P_DY, P_DZ, P_GAMMA, P_GZ, P_NU, P_ETA, P_KAPPA0, P_DIFFRHO,
  P_ETA_S, P_CHI_S, P_DIFFRHO_S, P_ZS, P_ZT, P_TAU_U, P_TAU_A, P_T_RAMP,
  P_FB, P_CADV, P_CDIFF, P_DT_FIXED, P_BEXT_X, P_BEXT_Y, P_BEXT_Z,
  P_NC_TAU, P_NC_LMAG, P_NC_LW, P_NC_ZMAX, P_NC_ZW, NPARAM
};

typedef struct {
  int nx, ny, nz, bcz;
  const double* p;
} grid_t;

static size_t ix(const grid_t* g, int f, int k, int j, int i) {
  size_t mx = (size_t)g->nx + 2 * NG, my = (size_t)g->ny + 2 * NG,
         mz = (size_t)g->nz + 2 * NG;
  return (((size_t)f * mz + (size_t)(k + NG)) * my + (size_t)(j + NG)) * mx +
         (size_t)(i + NG);
}

/* Sixth-order centred weights (Fornberg 1988): first derivative
 * [45(f1-f-1) - 9(f2-f-2) + (f3-f-3)]/(60h); second derivative
 * [2(f3+f-3) - 27(f2+f-2) + 270(f1+f-1) - 490 f0]/(180h^2). */
static const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
static const double W2[4] = {-490.0 / 180.0, 270.0 / 180.0, -27.0 / 180.0,
                             2.0 / 180.0};

static double spacing(const grid_t* g, int axis) {
  return axis == 0 ? g->p[P_DX] : axis == 1 ? g->p[P_DY] : g->p[P_DZ];
}

/* Vertical grid (the production grid's spacing grows from about 100 km in
 * the photosphere and chromosphere to about 800 km in the upper corona,
 * Sect. 1; the snapshots carry the inverse spacing dz_1, Sect. 5.3).  The
 * positions z_k of the layers k = -3 .. nz+2 are given (or_set_zgrid); the
 * layer index xi = k is the uniform coordinate, and with the sixth-order
 * index-space derivatives z' = D1_xi z, z'' = D2_xi z the chain rule gives
 *   df/dz = f_xi / z',  d2f/dz2 = f_xixi / z'^2 - f_xi z'' / z'^3.
 * Unset, z_k = k dz and the stencils divide by dz as before. */
static double* zg = NULL; /* z at k = -3 .. nz+2 */
static int zg_nz = -1;

void or_set_zgrid(int nz, const double* z) {
  free(zg);
  zg = NULL;
  zg_nz = -1;
  if (!z || nz <= 0) return;
  zg = (double*)malloc(sizeof(double) * (size_t)(nz + 2 * NG));
  memcpy(zg, z, sizeof(double) * (size_t)(nz + 2 * NG));
  zg_nz = nz;
}

static int zgrid_on(const grid_t* g) { return zg != NULL && zg_nz == g->nz; }

static double zpos(const grid_t* g, int k) { return zgrid_on(g) ? zg[k + NG] : (double)k * g->p[P_DZ]; }

/* dxi/dz and d2xi/dz2 at layer k (interior layers only: the stencil of z
 * reaches k +- 3) */
static void zmetric(const grid_t* g, int k, double* m1, double* m2) {
  double z1 = 0.0, z2 = 0.0;
  for (int m = 1; m <= 3; ++m) {
    z1 += W1[m] * (zpos(g, k + m) - zpos(g, k - m));
    z2 += W2[m] * (zpos(g, k + m) + zpos(g, k - m));
  }
  z2 += W2[0] * zpos(g, k);
  *m1 = 1.0 / z1;
  *m2 = -z2 / (z1 * z1 * z1);
}

/* value of field f at (i,j,k) displaced by m along `axis` */
static double at(const grid_t* g, const double* u, int f, int k, int j, int i,
                 int axis, int m) {
  if (axis == 0) i += m;
  else if (axis == 1) j += m;
  else k += m;
  return u[ix(g, f, k, j, i)];
}

static double d1(const grid_t* g, const double* u, int f, int k, int j, int i,
                 int axis) {
  double s = 0.0;
  for (int m = 1; m <= 3; ++m)
    s += W1[m] * (at(g, u, f, k, j, i, axis, m) - at(g, u, f, k, j, i, axis, -m));
  if (axis == 2 && zgrid_on(g)) {
    double m1, m2;
    zmetric(g, k, &m1, &m2);
    return s * m1;
  }
  return s / spacing(g, axis);
}

static double d2(const grid_t* g, const double* u, int f, int k, int j, int i,
                 int axis) {
  double s = W2[0] * u[ix(g, f, k, j, i)];
  for (int m = 1; m <= 3; ++m)
    s += W2[m] * (at(g, u, f, k, j, i, axis, m) + at(g, u, f, k, j, i, axis, -m));
  if (axis == 2 && zgrid_on(g)) {
    double s1 = 0.0, m1, m2;
    for (int m = 1; m <= 3; ++m)
      s1 += W1[m] * (at(g, u, f, k, j, i, axis, m) - at(g, u, f, k, j, i, axis, -m));
    zmetric(g, k, &m1, &m2);
    return s * m1 * m1 + s1 * m2;
  }
  double h = spacing(g, axis);
  return s / (h * h);
}

/* mixed derivative d_a d_b f = D1_a(D1_b f), the tensor product of the first
 * derivative weights, a != b */
static double d11(const grid_t* g, const double* u, int f, int k, int j, int i,
                  int a, int b) {
  double s = 0.0;
  for (int m = 1; m <= 3; ++m)
    for (int n = 1; n <= 3; ++n) {
      double acc = 0.0;
      for (int sm = -1; sm <= 1; sm += 2)
        for (int sn = -1; sn <= 1; sn += 2) {
          int d[3] = {0, 0, 0};
          d[a] += sm * m;
          d[b] += sn * n;
          acc += (double)(sm * sn) * u[ix(g, f, k + d[2], j + d[1], i + d[0])];
        }
      s += W1[m] * W1[n] * acc;
    }
  if ((a == 2 || b == 2) && zgrid_on(g)) {
    double m1, m2;
    zmetric(g, k, &m1, &m2);
    return s * m1 / spacing(g, a == 2 ? b : a);
  }
  return s / (spacing(g, a) * spacing(g, b));
}

/* Swamp weight w(z) (Sect. 4.3): cubic step from 0 at z_s to 1 at z_t with
 * zero slope at both ends; also returns dw/dz. */
void or_swamp_weight(const double* p, double z, double* w, double* wp) {
  double zs = p[P_ZS], zt = p[P_ZT];
  if (!(zt > zs)) { *w = 0.0; *wp = 0.0; return; }
  double s = (z - zs) / (zt - zs);
  if (s <= 0.0) { *w = 0.0; *wp = 0.0; return; }
  if (s >= 1.0) { *w = 1.0; *wp = 0.0; return; }
  *w = s * s * (3.0 - 2.0 * s);
  *wp = 6.0 * s * (1.0 - s) / (zt - zs);
}

/* ---------------------------------------------------------------------- */
/* Plain 2D discrete Fourier transform (separable sums, exact twiddle table)
 * used by the potential-field extrapolation (Sect. 4.2, Eqs. 16-17) and by
 * the inversion of the magnetogram into A_x, A_y (Sect. 2.4, Eq. 7). */

static void dft_axis(int n, int count, int stride_elem, int stride_line,
                     double* re, double* im, int sign) {
  double* cr = (double*)malloc(sizeof(double) * n);
  double* ci = (double*)malloc(sizeof(double) * n);
  for (int r = 0; r < n; ++r) {
    cr[r] = cos(2.0 * M_PI * (double)r / (double)n);
    ci[r] = (double)sign * sin(2.0 * M_PI * (double)r / (double)n);
  }
  /* lines are independent */
#pragma omp parallel for schedule(static)
  for (int l = 0; l < count; ++l) {
    double* tr = (double*)malloc(sizeof(double) * n);
    double* ti = (double*)malloc(sizeof(double) * n);
    double* xr = re + (size_t)l * stride_line;
    double* xi = im + (size_t)l * stride_line;
    for (int m = 0; m < n; ++m) {
      double sr = 0.0, si = 0.0;
      for (int x = 0; x < n; ++x) {
        int r = (int)(((long)m * x) % n);
        double ar = xr[(size_t)x * stride_elem], ai = xi[(size_t)x * stride_elem];
        sr += ar * cr[r] - ai * ci[r];
        si += ar * ci[r] + ai * cr[r];
      }
      tr[m] = sr;
      ti[m] = si;
    }
    for (int m = 0; m < n; ++m) {
      xr[(size_t)m * stride_elem] = tr[m];
      xi[(size_t)m * stride_elem] = ti[m];
    }
    free(tr);
    free(ti);
  }
  free(cr); free(ci);
}

/* forward (sign=-1) or unnormalised inverse (sign=+1) 2D DFT of ny x nx */
static void dft2(int nx, int ny, double* re, double* im, int sign) {
  dft_axis(nx, ny, 1, nx, re, im, sign);   /* along x, one line per y */
  dft_axis(ny, nx, nx, 1, re, im, sign);   /* along y, one line per x */
}

static double wavenumber(int m, int n, double len) {
  int mm = (2 * m > n) ? m - n : m;
  return 2.0 * M_PI * (double)mm / len;
}

/* Potential-field extrapolation of one horizontal plane (Eqs. 16-17):
 * out_j = IDFT( DFT(in) * exp(zfac[j] * |k|) ), j = 0..nout-1, where
 * zfac = -Delta''z for the upper boundary (decay with height) and
 * +f_b * Delta''z for the inverted extrapolation below the photosphere
 * (Sect. 2.4).  |k| uses the continuous wavenumbers 2 pi m / L. */
void or_pfe_plane(int nx, int ny, double lx, double ly, const double* in,
                  int nout, const double* zfac, double* out) {
  size_t n = (size_t)nx * ny;
  double* hr = (double*)malloc(sizeof(double) * n);
  double* hi = (double*)malloc(sizeof(double) * n);
  double* wr = (double*)malloc(sizeof(double) * n);
  double* wi = (double*)malloc(sizeof(double) * n);
  for (size_t q = 0; q < n; ++q) { hr[q] = in[q]; hi[q] = 0.0; }
  dft2(nx, ny, hr, hi, -1);
  for (int o = 0; o < nout; ++o) {
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) {
        double kx = wavenumber(a, nx, lx), ky = wavenumber(b, ny, ly);
        double mlt = exp(zfac[o] * sqrt(kx * kx + ky * ky));
        wr[(size_t)b * nx + a] = hr[(size_t)b * nx + a] * mlt;
        wi[(size_t)b * nx + a] = hi[(size_t)b * nx + a] * mlt;
      }
    dft2(nx, ny, wr, wi, +1);
    for (size_t q = 0; q < n; ++q) out[(size_t)o * n + q] = wr[q] / (double)n;
  }
  free(hr); free(hi); free(wr); free(wi);
}

/* modified wavenumber of the sixth-order first derivative:
 * D1 exp(i k x) = i kt exp(i k x), kt h = [45 sin(kh) - 9 sin(2kh) + sin(3kh)]/30;
 * zero for the Nyquist mode (2m = n) and the mean. */
static double kmod(int m, int n, double h) {
  if (m == 0 || 2 * m == n) return 0.0;
  double th = 2.0 * M_PI * (double)((2 * m > n) ? m - n : m) / (double)n;
  return (45.0 * sin(th) - 9.0 * sin(2.0 * th) + sin(3.0 * th)) / (30.0 * h);
}

/* Vector potential of the prescribed photospheric B_z (Eq. 7, Weyl gauge
 * A_z = 0): A^_x = i kt_y B^_z / kt^2, A^_y = -i kt_x B^_z / kt^2, modes with
 * kt^2 = 0 set to zero, so that D1_x A_y - D1_y A_x reproduces the band-limited
 * B_z exactly. */
void or_a_target(int nx, int ny, double dx, double dy, const double* bz,
                 double* ax, double* ay) {
  size_t n = (size_t)nx * ny;
  double* br = (double*)malloc(sizeof(double) * n);
  double* bi = (double*)malloc(sizeof(double) * n);
  double* xr = (double*)malloc(sizeof(double) * n);
  double* xi = (double*)malloc(sizeof(double) * n);
  double* yr = (double*)malloc(sizeof(double) * n);
  double* yi = (double*)malloc(sizeof(double) * n);
  for (size_t q = 0; q < n; ++q) { br[q] = bz[q]; bi[q] = 0.0; }
  dft2(nx, ny, br, bi, -1);
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) {
      size_t q = (size_t)b * nx + a;
      double kx = kmod(a, nx, dx), ky = kmod(b, ny, dy);
      double k2 = kx * kx + ky * ky;
      if (k2 == 0.0) { xr[q] = xi[q] = yr[q] = yi[q] = 0.0; continue; }
      /* i*ky*B/k2 */
      xr[q] = -ky * bi[q] / k2;
      xi[q] = ky * br[q] / k2;
      /* -i*kx*B/k2 */
      yr[q] = kx * bi[q] / k2;
      yi[q] = -kx * br[q] / k2;
    }
  dft2(nx, ny, xr, xi, +1);
  dft2(nx, ny, yr, yi, +1);
  for (size_t q = 0; q < n; ++q) { ax[q] = xr[q] / (double)n; ay[q] = yr[q] / (double)n; }
  free(br); free(bi); free(xr); free(xi); free(yr); free(yi);
}

/* ---------------------------------------------------------------------- */
/* Ghost filling (Sect. 2.4, 2.5, 4.1, 4.2).  Order: periodic x,y rims of the
 * layers that carry state, then the pointwise bottom/top rules over whole
 * padded planes, then the potential-field ghosts of A, then the rims of the
 * ghost layers. */

static void fill_rims(const grid_t* g, double* u, int f, int k) {
  int nx = g->nx, ny = g->ny;
  /* x rims of the interior rows, then y rims of whole padded rows (corners) */
  for (int j = 0; j < ny; ++j)
    for (int m = 0; m < NG; ++m) {
      u[ix(g, f, k, j, -1 - m)] = u[ix(g, f, k, j, nx - 1 - m)];
      u[ix(g, f, k, j, nx + m)] = u[ix(g, f, k, j, m)];
    }
  for (int m = 0; m < NG; ++m)
    for (int i = -NG; i < nx + NG; ++i) {
      u[ix(g, f, k, -1 - m, i)] = u[ix(g, f, k, ny - 1 - m, i)];
      u[ix(g, f, k, ny + m, i)] = u[ix(g, f, k, m, i)];
    }
}

static void fill_ghosts_impl(const int* dims, const double* p, double* u, const double* lnrho0, int do_pfe);

void or_fill_ghosts(const int* dims, const double* p, double* u, const double* lnrho0) {
  fill_ghosts_impl(dims, p, u, lnrho0, 1);
}

/* Every ghost rule except the potential-field extrapolation of A (for
 * planes too large for the plain DFT; the caller supplies those ghosts). */
void or_fill_ghosts_nopfe(const int* dims, const double* p, double* u, const double* lnrho0) {
  fill_ghosts_impl(dims, p, u, lnrho0, 0);
}

static void fill_ghosts_impl(const int* dims, const double* p, double* u, const double* lnrho0, int do_pfe) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  double dz = p[P_DZ], gz = p[P_GZ];

  /* (1) periodic rims of the layers that carry state */
  for (int f = 0; f < NFIELD; ++f)
    for (int k = 0; k < nz; ++k) fill_rims(g, u, f, k);
  if (g->bcz == 0)
    for (int k = -NG; k < 0; ++k) { fill_rims(g, u, F_UX, k); fill_rims(g, u, F_UY, k); }

  if (g->bcz == 1) {
    /* periodic in z: copies of the opposite interior layers */
    for (int f = 0; f < NFIELD; ++f)
      for (int m = 1; m <= NG; ++m)
        for (int j = -NG; j < ny + NG; ++j)
          for (int i = -NG; i < nx + NG; ++i) {
            u[ix(g, f, -m, j, i)] = u[ix(g, f, nz - m, j, i)];
            u[ix(g, f, nz - 1 + m, j, i)] = u[ix(g, f, m - 1, j, i)];
          }
    return;
  }

  /* (2) pointwise rules over the whole padded plane */
  for (int j = -NG; j < ny + NG; ++j)
    for (int i = -NG; i < nx + NG; ++i) {
      /* bottom: ln rho fixed to the initial profile at and below the
       * photosphere (Sect. 2.5, 'fg'); */
      for (int m = 1; m <= NG; ++m) u[ix(g, F_LNRHO, -m, j, i)] = lnrho0[NG - m];
      /* ln T from hydrostatic equilibrium, recursively downward (Eq. 8, read
       * with p = rho T, i.e. the c_v/c_p factor taken as 1):
       * p_j = p_{j+1} exp(-dz g_z / T_{j+1}) */
      for (int m = 1; m <= NG; ++m) {
        double th1 = u[ix(g, F_LNTT, -m + 1, j, i)];
        double l1 = u[ix(g, F_LNRHO, -m + 1, j, i)];
        double l0 = u[ix(g, F_LNRHO, -m, j, i)];
        double dzl = zgrid_on(g) ? zpos(g, -m + 1) - zpos(g, -m) : dz;
        u[ix(g, F_LNTT, -m, j, i)] = th1 + l1 - l0 - dzl * gz / exp(th1);
      }
      /* closed bottom: u_z antisymmetric about the photosphere (u_z = 0 there) */
      for (int m = 1; m <= NG; ++m) u[ix(g, F_UZ, -m, j, i)] = -u[ix(g, F_UZ, m, j, i)];

      /* top: ln T symmetric (Eq. 11) */
      int kt = nz - 1;
      for (int m = 1; m <= NG; ++m) u[ix(g, F_LNTT, kt + m, j, i)] = u[ix(g, F_LNTT, kt - m, j, i)];
      /* ln rho hydrostatic with the boundary temperature (Eq. 13, read with
       * signed g_z < 0 and p = rho T): rho_{nz+j} = rho_{nz-j} exp((z_{nz+j} -
       * z_{nz-j}) g_z / T_nz) */
      double ttop = exp(u[ix(g, F_LNTT, kt, j, i)]);
      for (int m = 1; m <= NG; ++m) {
        double span = zgrid_on(g) ? zpos(g, kt + m) - zpos(g, kt - m) : 2.0 * m * dz;
        u[ix(g, F_LNRHO, kt + m, j, i)] = u[ix(g, F_LNRHO, kt - m, j, i)] + span * gz / ttop;
      }
      /* closed top: u_z antisymmetric, horizontal velocity symmetric */
      for (int m = 1; m <= NG; ++m) {
        u[ix(g, F_UZ, kt + m, j, i)] = -u[ix(g, F_UZ, kt - m, j, i)];
        u[ix(g, F_UX, kt + m, j, i)] = u[ix(g, F_UX, kt - m, j, i)];
        u[ix(g, F_UY, kt + m, j, i)] = u[ix(g, F_UY, kt - m, j, i)];
      }
    }

  /* (3) potential-field ghosts of all three components of A: regular
   * extrapolation upward (Eq. 17, Delta''z = z_{nz-1+m} - z_{nz-1}, m dz on
   * the uniform grid), inverted extrapolation downward over z_0 - z_{-m}
   * with the contrast growth reduced by f_b (Sect. 2.4). */
  if (!do_pfe) return;
  size_t n = (size_t)nx * ny;
  double* plane = (double*)malloc(sizeof(double) * n);
  double* gh = (double*)malloc(sizeof(double) * n * NG);
  double lx = nx * p[P_DX], ly = ny * p[P_DY];
  for (int side = 0; side < 2; ++side) {
    int kb = side == 0 ? nz - 1 : 0;
    double zf[NG];
    for (int m = 1; m <= NG; ++m) {
      if (zgrid_on(g)) {
        double d = side == 0 ? zpos(g, kb + m) - zpos(g, kb) : zpos(g, kb) - zpos(g, kb - m);
        zf[m - 1] = side == 0 ? -d : p[P_FB] * d;
      } else {
        zf[m - 1] = side == 0 ? -(double)m * dz : p[P_FB] * (double)m * dz;
      }
    }
    for (int f = F_AX; f <= F_AZ; ++f) {
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) plane[(size_t)j * nx + i] = u[ix(g, f, kb, j, i)];
      or_pfe_plane(nx, ny, lx, ly, plane, NG, zf, gh);
      for (int m = 1; m <= NG; ++m) {
        int kg = side == 0 ? kb + m : kb - m;
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i)
            u[ix(g, f, kg, j, i)] = gh[(size_t)(m - 1) * n + (size_t)j * nx + i];
      }
    }
  }
  free(plane);
  free(gh);

  /* (4) rims of all ghost layers */
  for (int f = 0; f < NFIELD; ++f)
    for (int m = 1; m <= NG; ++m) { fill_rims(g, u, f, -m); fill_rims(g, u, f, nz - 1 + m); }
}

/* ---------------------------------------------------------------------- */
/* Driver: two snapshots v0 (time t0) and v1 (t1) interpolated linearly in
 * time (Sect. 2.3, two-step driver scheme), times the linear switch-on ramp
 * r(t) = min(t / t_ramp, 1) (Sect. 2.3, first minute of the run). */
static void driver_weights(const double* p, double t0, double t1, double t,
                           double* r, double* s) {
  double tr = p[P_T_RAMP];
  *r = tr > 0.0 ? (t / tr < 0.0 ? 0.0 : (t / tr > 1.0 ? 1.0 : t / tr)) : 1.0;
  double q = t1 > t0 ? (t - t0) / (t1 - t0) : 0.0;
  *s = q < 0.0 ? 0.0 : (q > 1.0 ? 1.0 : q);
}

/* Right-hand side of the four evolution equations at interior cells
 * (k in [k_lo, k_hi)); rows of the stateful horizontal-velocity ghost layers
 * below the photosphere carry only the nudging term (Eq. 5 applied at
 * j in {0,-1,-2,-3}).  Equations (ln-variable resistive MHD, mu0 = 1,
 * p = rho T, Weyl gauge; see the scheme):
 *  dA/dt = u x B - eta J + eta_s w lap A + e_z eta_s w' div A       (Eq. 18)
 *          - tau_A (A_hor - A_target) at the photosphere           (Sect. 2.1)
 *  du/dt = -(u.grad)u - T (grad ln rho + grad ln T) + g_z e_z + J x B / rho
 *          + nu (lap u + grad div u / 3 + 2 S.grad ln rho)
 *          - tau_u (u_hor - r v*) at the photosphere               (Eq. 5)
 *  dlnrho/dt = -u.grad ln rho - div u + D_rho (lap ln rho + |grad ln rho|^2)
 *          + chi_rho w lap ln rho                                   (Eq. 20)
 *  dlnT/dt = -u.grad ln T - (gamma-1) div u + (gamma-1)(eta J^2 + 2 rho nu S^2)/(rho T)
 *          + (gamma-1) kappa0 T^{5/2}/rho (lap ln T + 3.5 |grad ln T|^2)
 *          + chi_s w lap ln T                                       (Eq. 19)
 *  photosphere: dlnrho/dt = 0 (density held at its initial profile,
 *  Sect. 2.5), du_z/dt = 0 (closed); top layer: du_z/dt = 0 (Sect. 4). */
/* ---- Newtonian cooling (Sect. 3.1, Eqs. 9-10) -------------------------
 * Read as a relaxation of ln T: d ln T/dt += -tau (1 - T* / T) c_rho c_z,
 * T* = sqrt(T0(z) T'(rho)), with T'(rho) the initial temperature T0(z') at
 * the height z' where the initial density rho0(z') equals the local rho.
 * The initial profiles over the interior layers are set once by
 * or_set_nc_profile (arrays of nz + 6 entries, ghost layers included). */
static double* nc_lr = NULL; /* ln rho0 at layers 0 .. nz-1 */
static double* nc_lt = NULL; /* ln T0 at layers 0 .. nz-1 */
static int nc_nz = 0;

void or_set_nc_profile(int nz, const double* lnrho0, const double* lnT0) {
  free(nc_lr);
  free(nc_lt);
  nc_lr = (double*)malloc(sizeof(double) * nz);
  nc_lt = (double*)malloc(sizeof(double) * nz);
  for (int k = 0; k < nz; ++k) {
    nc_lr[k] = lnrho0[NG + k];
    nc_lt[k] = lnT0[NG + k];
  }
  nc_nz = nz;
}

/* ln T'(rho): walk up the layers to the first segment [m, m+1] whose initial
 * ln rho brackets L and interpolate ln T0 linearly there; below the bottom
 * value or above the top one, the end layers. */
static double nc_lnT_prime(double L) {
  if (L >= nc_lr[0]) return nc_lt[0];
  if (L <= nc_lr[nc_nz - 1]) return nc_lt[nc_nz - 1];
  for (int m = 0; m + 1 < nc_nz; ++m) {
    if (L <= nc_lr[m] && L >= nc_lr[m + 1]) {
      double s = (L - nc_lr[m]) / (nc_lr[m + 1] - nc_lr[m]);
      return nc_lt[m] + s * (nc_lt[m + 1] - nc_lt[m]);
    }
  }
  return nc_lt[nc_nz - 1];
}

/* 1 up to x1 - w, 0 from x1 on, half a cosine period between */
static double nc_cutoff(double x, double x1, double w) {
  if (x <= x1 - w) return 1.0;
  if (x >= x1) return 0.0;
  return 0.5 * (1.0 + cos(M_PI * (x - (x1 - w)) / w));
}

/* z: the height of layer k */
static double nc_term(const double* p, int k, double z, double lnrho, double lnT) {
  double cz = nc_cutoff(z, p[P_NC_ZMAX], p[P_NC_ZW]);
  double crho = nc_cutoff(nc_lr[0] - lnrho, p[P_NC_LMAG], p[P_NC_LW]);
  double lnTstar = 0.5 * (nc_lt[k] + nc_lnT_prime(lnrho));
  return -p[P_NC_TAU] * (1.0 - exp(lnTstar - lnT)) * crho * cz;
}

/* Right-hand side at one interior cell (k, j, i); out[8] in field order.
 * r, s: ramp and driver interpolation weight at the evaluation time. */
static void rhs_cell(const grid_t* g, const double* u, const double* axt, const double* ayt,
                     const double* v0, const double* v1, double r, double s, int k, int j, int i,
                     double* out) {
  const double* p = g->p;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  double gam = p[P_GAMMA], gz = p[P_GZ], nu = p[P_NU], eta = p[P_ETA];
  double kap = p[P_KAPPA0], drho = p[P_DIFFRHO];
  double eta_s = p[P_ETA_S], chi_s = p[P_CHI_S], drho_s = p[P_DIFFRHO_S];
  double w = 0.0, wp = 0.0;
  or_swamp_weight(p, zpos(g, k), &w, &wp);
  double A[3], U[3], D1A[3][3], D1U[3][3], lapA[3], lapU[3];
  double gdA[3], gdU[3], gL[3], gT[3];
  for (int c = 0; c < 3; ++c) {
    A[c] = u[ix(g, F_AX + c, k, j, i)];
    U[c] = u[ix(g, F_UX + c, k, j, i)];
    lapA[c] = lapU[c] = 0.0;
    for (int a = 0; a < 3; ++a) {
      D1A[c][a] = d1(g, u, F_AX + c, k, j, i, a); /* d_a A_c */
      D1U[c][a] = d1(g, u, F_UX + c, k, j, i, a); /* d_a u_c */
      lapA[c] += d2(g, u, F_AX + c, k, j, i, a);
      lapU[c] += d2(g, u, F_UX + c, k, j, i, a);
    }
  }
  /* grad(div A)_a = sum_c d_a d_c A_c, with d_a d_a the second
   * derivative and d_a d_c (a != c) the mixed one */
  for (int a = 0; a < 3; ++a) {
    gdA[a] = gdU[a] = 0.0;
    for (int c = 0; c < 3; ++c) {
      if (c == a) {
        gdA[a] += d2(g, u, F_AX + c, k, j, i, a);
        gdU[a] += d2(g, u, F_UX + c, k, j, i, a);
      } else {
        gdA[a] += d11(g, u, F_AX + c, k, j, i, a, c);
        gdU[a] += d11(g, u, F_UX + c, k, j, i, a, c);
      }
    }
  }
  double lapL = 0.0, lapT = 0.0;
  for (int a = 0; a < 3; ++a) {
    gL[a] = d1(g, u, F_LNRHO, k, j, i, a);
    gT[a] = d1(g, u, F_LNTT, k, j, i, a);
    lapL += d2(g, u, F_LNRHO, k, j, i, a);
    lapT += d2(g, u, F_LNTT, k, j, i, a);
  }
  double lnrho = u[ix(g, F_LNRHO, k, j, i)], lnT = u[ix(g, F_LNTT, k, j, i)];
  double rho = exp(lnrho), T = exp(lnT);

  double B[3] = {D1A[2][1] - D1A[1][2] + p[P_BEXT_X],
                 D1A[0][2] - D1A[2][0] + p[P_BEXT_Y],
                 D1A[1][0] - D1A[0][1] + p[P_BEXT_Z]};
  double J[3];
  for (int a = 0; a < 3; ++a) J[a] = gdA[a] - lapA[a];
  double divA = D1A[0][0] + D1A[1][1] + D1A[2][2];
  double divU = D1U[0][0] + D1U[1][1] + D1U[2][2];

  /* induction */
  double uxB[3] = {U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2],
                   U[0] * B[1] - U[1] * B[0]};
  double dA[3];
  for (int a = 0; a < 3; ++a) dA[a] = uxB[a] - eta * J[a] + eta_s * w * lapA[a];
  dA[2] += eta_s * wp * divA;

  /* momentum */
  double JxB[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2],
                   J[0] * B[1] - J[1] * B[0]};
  double S[3][3], S2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      S[a][b] = 0.5 * (D1U[a][b] + D1U[b][a]) - (a == b ? divU / 3.0 : 0.0);
      S2 += S[a][b] * S[a][b];
    }
  double dU[3];
  for (int a = 0; a < 3; ++a) {
    double adv = 0.0, SgL = 0.0;
    for (int b = 0; b < 3; ++b) {
      adv += U[b] * D1U[a][b];
      SgL += S[a][b] * gL[b];
    }
    dU[a] = -adv - T * (gL[a] + gT[a]) + JxB[a] / rho +
            nu * (lapU[a] + gdU[a] / 3.0 + 2.0 * SgL);
  }
  dU[2] += gz;

  /* continuity */
  double ugL = U[0] * gL[0] + U[1] * gL[1] + U[2] * gL[2];
  double gL2 = gL[0] * gL[0] + gL[1] * gL[1] + gL[2] * gL[2];
  double dL = -ugL - divU + drho * (lapL + gL2) + drho_s * w * lapL;

  /* energy (ln T) */
  double ugT = U[0] * gT[0] + U[1] * gT[1] + U[2] * gT[2];
  double gT2 = gT[0] * gT[0] + gT[1] * gT[1] + gT[2] * gT[2];
  double J2 = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
  double heat = (gam - 1.0) * (eta * J2 + 2.0 * rho * nu * S2) / (rho * T);
  double cond = (gam - 1.0) * kap * pow(T, 2.5) / rho * (lapT + 3.5 * gT2);
  double dTh = -ugT - (gam - 1.0) * divU + heat + cond + chi_s * w * lapT;
  if (p[P_NC_TAU] > 0.0 && g->bcz == 0) dTh += nc_term(p, k, zpos(g, k), lnrho, lnT);

  if (g->bcz == 0) {
    if (k == 0) {
      double vx = v0[(size_t)j * nx + i] + s * (v1[(size_t)j * nx + i] - v0[(size_t)j * nx + i]);
      double vy = v0[(size_t)nx * ny + (size_t)j * nx + i] +
                  s * (v1[(size_t)nx * ny + (size_t)j * nx + i] - v0[(size_t)nx * ny + (size_t)j * nx + i]);
      dA[0] -= p[P_TAU_A] * (A[0] - axt[(size_t)j * nx + i]);
      dA[1] -= p[P_TAU_A] * (A[1] - ayt[(size_t)j * nx + i]);
      dU[0] -= p[P_TAU_U] * (U[0] - r * vx);
      dU[1] -= p[P_TAU_U] * (U[1] - r * vy);
      dU[2] = 0.0;
      dL = 0.0;
    }
    if (k == nz - 1) dU[2] = 0.0;
  }
  out[0] = dA[0]; out[1] = dA[1]; out[2] = dA[2];
  out[3] = dU[0]; out[4] = dU[1]; out[5] = dU[2];
  out[6] = dL; out[7] = dTh;
}

void or_rhs(const int* dims, const double* p, const double* u,
            const double* axt, const double* ayt, const double* v0,
            const double* v1, double t0, double t1, double t, double* rhs) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  double r, s;
  driver_weights(p, t0, t1, t, &r, &s);

#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double o8[8];
        rhs_cell(g, u, axt, ayt, v0, v1, r, s, k, j, i, o8);
        for (int f = 0; f < NFIELD; ++f) rhs[ix(g, f, k, j, i)] = o8[f];
      }

  if (g->bcz == 0) {
    /* ghost layers of u_hor below the photosphere: nudging only (Eq. 5) */
    for (int m = 1; m <= NG; ++m)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          size_t q = (size_t)j * nx + i, n2 = (size_t)nx * ny;
          double vx = v0[q] + s * (v1[q] - v0[q]);
          double vy = v0[n2 + q] + s * (v1[n2 + q] - v0[n2 + q]);
          rhs[ix(g, F_UX, -m, j, i)] = -p[P_TAU_U] * (u[ix(g, F_UX, -m, j, i)] - r * vx);
          rhs[ix(g, F_UY, -m, j, i)] = -p[P_TAU_U] * (u[ix(g, F_UY, -m, j, i)] - r * vy);
        }
  }
}

/* Right-hand side at a list of cells: cells[3 c + 0..2] = (k, j, i);
 * out[8 c + f].  Same arithmetic as or_rhs, for sampled checks of large
 * grids. */
void or_rhs_cells(const int* dims, const double* p, const double* u, const double* axt,
                  const double* ayt, const double* v0, const double* v1, double t0, double t1,
                  double t, int ncell, const int* cells, double* out) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  double r, s;
  driver_weights(p, t0, t1, t, &r, &s);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < ncell; ++c)
    rhs_cell(&G, u, axt, ayt, v0, v1, r, s, cells[3 * c], cells[3 * c + 1], cells[3 * c + 2], out + 8 * c);
}

/* Magnetic field B = curl A + B_ext at an interior cell (Eq. 6). */
static void bfield(const grid_t* g, const double* u, int k, int j, int i, double* B) {
  B[0] = d1(g, u, F_AZ, k, j, i, 1) - d1(g, u, F_AY, k, j, i, 2) + g->p[P_BEXT_X];
  B[1] = d1(g, u, F_AX, k, j, i, 2) - d1(g, u, F_AZ, k, j, i, 0) + g->p[P_BEXT_Y];
  B[2] = d1(g, u, F_AY, k, j, i, 0) - d1(g, u, F_AX, k, j, i, 1) + g->p[P_BEXT_Z];
}

/* CFL time step from the ghost-filled state: the smaller of
 * C_adv / max(sum|u_i|/dx_i + sqrt(gamma T + B^2/rho) sqrt(sum 1/dx_i^2)) and
 * C_diff / max(D_max sum 1/dx_i^2), D_max the largest diffusivity of the cell. */
double or_cfl(const int* dims, const double* p, const double* u) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  double dx = p[P_DX], dy = p[P_DY], dz = p[P_DZ];
  double gam = p[P_GAMMA];
  double max_adv = 0.0, max_dif = 0.0;
  for (int k = 0; k < g->nz; ++k) {
    /* the local vertical spacing 1 / (dxi/dz) on a non-uniform grid */
    double dzk = dz;
    if (zgrid_on(g)) {
      double m1, m2;
      zmetric(g, k, &m1, &m2);
      dzk = 1.0 / m1;
    }
    double inv2 = 1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dzk * dzk);
    double w = 0.0, wp = 0.0;
    or_swamp_weight(p, zpos(g, k), &w, &wp);
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double B[3];
        bfield(g, u, k, j, i, B);
        double rho = exp(u[ix(g, F_LNRHO, k, j, i)]);
        double T = exp(u[ix(g, F_LNTT, k, j, i)]);
        double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        double adv = fabs(u[ix(g, F_UX, k, j, i)]) / dx + fabs(u[ix(g, F_UY, k, j, i)]) / dy +
                     fabs(u[ix(g, F_UZ, k, j, i)]) / dzk + sqrt(gam * T + B2 / rho) * sqrt(inv2);
        double dm = p[P_NU];
        double c1 = p[P_ETA] + p[P_ETA_S] * w;
        double c2 = p[P_DIFFRHO] + p[P_DIFFRHO_S] * w;
        double c3 = p[P_CHI_S] * w + (gam - 1.0) * p[P_KAPPA0] * pow(T, 2.5) / rho;
        if (c1 > dm) dm = c1;
        if (c2 > dm) dm = c2;
        if (c3 > dm) dm = c3;
        if (adv > max_adv) max_adv = adv;
        if (dm * inv2 > max_dif) max_dif = dm * inv2;
      }
  }
  double dt1 = max_adv > 0.0 ? p[P_CADV] / max_adv : INFINITY;
  double dt2 = max_dif > 0.0 ? p[P_CDIFF] / max_dif : INFINITY;
  return dt1 < dt2 ? dt1 : dt2;
}

/* Global diagnostics of the ghost-filled state, FP64 sums in plain order:
 * out[0] E_kin = sum rho u^2/2 dV, out[1] E_mag = sum B^2/2 dV,
 * out[2] E_th = sum rho T/(gamma-1) dV, out[3] mass = sum rho dV,
 * out[4] net photospheric flux sum B_z(k=0) dx dy (zero for the flux-balanced
 * magnetograms of Sect. 2.1), out[5] unsigned flux sum |B_z(k=0)| dx dy,
 * out[6] max |div B| (identically zero for B = curl A, Eq. 6). */
void or_stats(const int* dims, const double* p, const double* u, double* out) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  double dx = p[P_DX], dy = p[P_DY], dz = p[P_DZ];
  double ek = 0, em = 0, eth = 0, ms = 0, fn = 0, fa = 0, dbm = 0;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  for (int k = 0; k < nz; ++k) {
    /* cell volume dx dy Delta'z, Delta'z = (z_{k+1} - z_{k-1}) / 2 the
     * vertical extent of the cell (Sect. 4.1); dz on the uniform grid */
    double dv = dx * dy * dz, m1 = 1.0 / dz, m2;
    if (zgrid_on(g)) {
      dv = dx * dy * 0.5 * (zpos(g, k + 1) - zpos(g, k - 1));
      zmetric(g, k, &m1, &m2);
    }
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double B[3];
        bfield(g, u, k, j, i, B);
        double rho = exp(u[ix(g, F_LNRHO, k, j, i)]);
        double T = exp(u[ix(g, F_LNTT, k, j, i)]);
        double ux = u[ix(g, F_UX, k, j, i)], uy = u[ix(g, F_UY, k, j, i)], uz = u[ix(g, F_UZ, k, j, i)];
        ek += 0.5 * rho * (ux * ux + uy * uy + uz * uz) * dv;
        em += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) * dv;
        eth += rho * T / (p[P_GAMMA] - 1.0) * dv;
        ms += rho * dv;
        if (k == 0) { fn += B[2] * dx * dy; fa += fabs(B[2]) * dx * dy; }
        /* div B = D1_x B_x + D1_y B_y + D1_z B_z with B from the same
         * stencils; B_x carries no x derivative, B_y no y derivative and B_z
         * no z derivative, so every value used lies inside the ghost zone */
        double divb = 0.0;
        for (int m = 1; m <= 3; ++m) {
          double bxp = d1(g, u, F_AZ, k, j, i + m, 1) - d1(g, u, F_AY, k, j, i + m, 2);
          double bxm = d1(g, u, F_AZ, k, j, i - m, 1) - d1(g, u, F_AY, k, j, i - m, 2);
          double byp = d1(g, u, F_AX, k, j + m, i, 2) - d1(g, u, F_AZ, k, j + m, i, 0);
          double bym = d1(g, u, F_AX, k, j - m, i, 2) - d1(g, u, F_AZ, k, j - m, i, 0);
          double bzp = d1(g, u, F_AY, k + m, j, i, 0) - d1(g, u, F_AX, k + m, j, i, 1);
          double bzm = d1(g, u, F_AY, k - m, j, i, 0) - d1(g, u, F_AX, k - m, j, i, 1);
          divb += W1[m] * ((bxp - bxm) / dx + (byp - bym) / dy +
                           (zgrid_on(g) ? (bzp - bzm) * m1 : (bzp - bzm) / dz));
        }
        if (fabs(divb) > dbm) dbm = fabs(divb);
      }
  }
  out[0] = ek; out[1] = em; out[2] = eth; out[3] = ms; out[4] = fn; out[5] = fa; out[6] = dbm;
}

/* ---------------------------------------------------------------------- */
/* One or more low-storage third-order Runge-Kutta steps (Williamson 1980,
 * 2N storage): df <- alpha_s df + dt RHS(f, t + c_s dt); f <- f + beta_s df,
 * alpha = (0, -5/9, -153/128), beta = (1/3, 15/16, 8/15), c = (0, 1/3, 3/4).
 * dt from the CFL rule of the state at the first substep (or dt_fixed > 0).
 * `u` is the padded state including the stateful horizontal-velocity ghosts
 * below the photosphere; `t` is advanced; dts (nullable) receives each dt. */
int or_run(const int* dims, const double* p, double* u, const double* lnrho0,
           const double* axt, const double* ayt, const double* v0, const double* v1,
           double t0, double t1, double* t, int nsteps, double* dts) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  size_t ntot = (size_t)NFIELD * (g->nx + 2 * NG) * (g->ny + 2 * NG) * (g->nz + 2 * NG);
  static const double alpha[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
  static const double beta[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
  static const double csub[3] = {0.0, 1.0 / 3.0, 3.0 / 4.0};
  double* df = (double*)calloc(ntot, sizeof(double));
  double* rhs = (double*)calloc(ntot, sizeof(double));
  if (!df || !rhs) { free(df); free(rhs); return -1; }
  for (int n = 0; n < nsteps; ++n) {
    double dt = 0.0;
    for (int sub = 0; sub < 3; ++sub) {
      or_fill_ghosts(dims, p, u, lnrho0);
      if (sub == 0) dt = p[P_DT_FIXED] > 0.0 ? p[P_DT_FIXED] : or_cfl(dims, p, u);
      memset(rhs, 0, ntot * sizeof(double));
      or_rhs(dims, p, u, axt, ayt, v0, v1, t0, t1, *t + csub[sub] * dt, rhs);
      /* update the cells that carry state: interior, plus the u_hor ghosts
       * below the photosphere */
      for (int f = 0; f < NFIELD; ++f)
        for (int k = -NG; k < g->nz; ++k) {
          if (k < 0 && !(g->bcz == 0 && (f == F_UX || f == F_UY))) continue;
          for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
              size_t q = ix(g, f, k, j, i);
              df[q] = alpha[sub] * df[q] + dt * rhs[q];
              u[q] = u[q] + beta[sub] * df[q];
            }
        }
    }
    *t += dt;
    if (dts) dts[n] = dt;
  }
  free(df);
  free(rhs);
  return 0;
}

/* Stencil probes for the pins: derivative `kind` (0: D1 along a, 1: D2 along
 * a, 2: D_a D_b) of field f at every interior cell, written to out
 * [nz][ny][nx]. */
void or_deriv(const int* dims, const double* p, const double* u, int f, int kind,
              int a, int b, double* out) {
  grid_t G = {dims[0], dims[1], dims[2], dims[3], p};
  const grid_t* g = &G;
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double v = kind == 0 ? d1(g, u, f, k, j, i, a)
                 : kind == 1 ? d2(g, u, f, k, j, i, a)
                             : d11(g, u, f, k, j, i, a, b);
        out[((size_t)k * g->ny + j) * g->nx + i] = v;
      }
}
