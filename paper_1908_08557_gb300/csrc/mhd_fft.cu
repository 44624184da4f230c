// mhd_fft.cu -- FP64 horizontal FFT of the potential-field boundary
// (Sect. 4.2, Eqs. 16-17; Sect. 2.4 inverted extrapolation) and of the
// magnetogram inversion (Sect. 2.4, Eq. 7).
//
// The six real boundary planes (A_x, A_y, A_z at the top layer and at the
// photosphere) travel as three complex planes:
//   P0 = A_x(top) + i A_y(top),  P1 = A_x(bot) + i A_y(bot),
//   P2 = A_z(top) + i A_z(bot).
// The extrapolation multiplier M(k) is real and even in k, so applying it to
// a packed plane extrapolates both real parts at once.  P2 carries two planes
// with different multipliers M_t, M_b; with F = FFT(P2) the spectrum to invert
// is a F(k) + b conj(F(-k)), a = (M_t + M_b)/2, b = (M_t - M_b)/2, whose inverse
// has real part = top ghost and imaginary part = bottom ghost.
//
// Kernels (radix-4 Stockham autosort in shared memory, FP64):
//   1. rows_fwd: pack rows from the state, FFT along x, store transposed
//   2. cols:     FFT along y, for each ghost layer j = 1..3 form the
//                extrapolated spectrum (M_t = exp(-|k| j dz),
//                M_b = exp(+f_b |k| j dz)), inverse FFT along y
//   3. rows_inv: inverse FFT along x, write real/imaginary parts into the
//                ghost layers (with their periodic x,y images)
#include "mhd_internal.h"

namespace mhd {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// nb lines of n = 2^logn complex points in a (b is scratch of equal size).
// Stockham autosort, radix 4, with one radix-2 stage first when logn is odd.
// With p the length of the sub-transforms done so far, radix-4 butterfly
// i in [0, n/4) has k = i mod p, j = i div p; it takes x[i + m n/4]
// (m = 0..3) times w^(m k), w = exp(-+2 pi i / (4p)), and writes their
// 4-point DFT c_q to y[4 j p + k + q p] = y[4i - 3k + q p].  At p = 1 every
// k is 0 and the twiddles drop out; the radix-2 stage (p = 1) writes
// x[i] +- x[i + n/2] to y[2i], y[2i + 1].  Returns the buffer holding the
// (unnormalised) transform.
__device__ double2* fft_lines(double2* a, double2* b, int n, int logn, int nb, const double2* __restrict__ tw,
                              bool inverse) {
  int p = 1, lp = 0;
  if (logn & 1) {
    const int half = n >> 1;
    const int total = nb * half;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int line = q >> (logn - 1);
      const int i = q & (half - 1);
      const double2 u0 = a[line * n + i], u1 = a[line * n + i + half];
      b[line * n + 2 * i] = cadd(u0, u1);
      b[line * n + 2 * i + 1] = csub(u0, u1);
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
    p = 2;
    lp = 1;
  }
  const int quarter = n >> 2;
  const int total = nb * quarter;
  for (; p < n; p <<= 2, lp += 2) {
    const int tws = logn - 2 - lp;  // twiddle index m k n / (4p) = (m k) << tws
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int line = q >> (logn - 2);
      const int i = q & (quarter - 1);
      const int k = i & (p - 1);
      const double2* x = a + line * n + i;
      double2 b0 = x[0], b1 = x[quarter], b2 = x[2 * quarter], b3 = x[3 * quarter];
      if (p > 1) {
        double2 w1 = __ldg(tw + (k << tws)), w2 = __ldg(tw + ((2 * k) << tws)), w3 = __ldg(tw + ((3 * k) << tws));
        if (inverse) {
          w1.y = -w1.y;
          w2.y = -w2.y;
          w3.y = -w3.y;
        }
        b1 = cmul(w1, b1);
        b2 = cmul(w2, b2);
        b3 = cmul(w3, b3);
      }
      const double2 t0 = cadd(b0, b2), t1 = csub(b0, b2), t2 = cadd(b1, b3), t3 = csub(b1, b3);
      // -i t3 for the forward transform, +i t3 for the inverse
      const double2 r3 = inverse ? make_double2(-t3.y, t3.x) : make_double2(t3.y, -t3.x);
      double2* y = b + line * n + 4 * i - 3 * k;
      y[0] = cadd(t0, t2);
      y[p] = cadd(t1, r3);
      y[2 * p] = csub(t0, t2);
      y[3 * p] = csub(t1, r3);
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// ---------------------------------------------------------------------------
// 1. forward rows.  mode 0: three boundary planes of the state; mode 1: one
// real plane `src2d` ([ny][nx], the magnetogram).
// mode 2 (adjoint of the potential-field ghosts): plane p = 3c + m - 1 packs
// the ghost adjoints of A_c at the top layer nz-1+m (real) and at -m
// (imaginary); mode 3: the complex plane dre + i dim (FP64 inputs).
template <typename R>
__global__ void __launch_bounds__(256) rows_fwd_kernel(FFTPlan fp, Layout L, const R* __restrict__ f,
                                                       const R* __restrict__ src2d, int mode,
                                                       const StepState* ss, int nb, const double* __restrict__ dre,
                                                       const double* __restrict__ dim) {
  extern __shared__ double2 sm[];
  if (ss && halted(ss)) return;
  const int nx = fp.nx, ny = fp.ny;
  const int y0 = blockIdx.x * nb;
  const int p = fp.p0 + blockIdx.y;
  double2* a = sm;
  double2* b = sm + nb * nx;
  const int kt = L.nz - 1;
  for (int q = threadIdx.x; q < nb * nx; q += blockDim.x) {
    const int line = q / nx, x = q - line * nx, y = y0 + line;
    double re, im;
    if (mode == 1) {
      re = (double)src2d[(long long)y * nx + x];
      im = 0.0;
    } else if (mode == 2) {
      const int cc = p / 3, m = p - 3 * cc + 1;
      re = (double)f[L.at(AX + cc, kt + m, y, x)];
      im = (double)f[L.at(AX + cc, -m, y, x)];
    } else if (mode == 3) {
      re = dre[(long long)y * nx + x];
      im = dim[(long long)y * nx + x];
    } else if (p == 0) {
      re = (double)f[L.at(AX, kt, y, x)];
      im = (double)f[L.at(AY, kt, y, x)];
    } else if (p == 1) {
      re = (double)f[L.at(AX, 0, y, x)];
      im = (double)f[L.at(AY, 0, y, x)];
    } else {
      re = (double)f[L.at(AZ, kt, y, x)];
      im = (double)f[L.at(AZ, 0, y, x)];
    }
    a[line * nx + x] = make_double2(re, im);
  }
  __syncthreads();
  double2* r = fft_lines(a, b, nx, fp.lognx, nb, fp.twx, false);
  // transposed store: P[p][x][y], consecutive threads walk y
  for (int q = threadIdx.x; q < nb * nx; q += blockDim.x) {
    const int x = q / nb, line = q - x * nb;
    fp.P[((long long)p * nx + x) * ny + y0 + line] = r[line * nx + x];
  }
}

// ---------------------------------------------------------------------------
// 2. columns.  A block owns column pairs (kx, nx - kx); both columns of a pair
// are needed to split the packed plane P2 (F(-k) lives in the mirror column).
// mode 0: potential-field extrapolation, 3 layers; mode 1: magnetogram
// inversion (Eq. 7): A^_x + i A^_y = (kt_x + i kt_y) B^_z / kt^2; mode 2: its
// transpose; mode 4: the filtered rotational part of the granulation field
// (Sect. 2.3, Eq. 3).  The spectra of lg output layers at a time are formed and
// inverted as one batch of lines, so each stage of the inverse transform has
// lg times the butterflies between two barriers; lg = nout needs two buffers
// of lg layers (the forward spectrum's buffer becomes the scratch), lg < nout
// three (the spectrum is kept).
__global__ void __launch_bounds__(256) cols_kernel(FFTPlan fp, int mode, const StepState* ss, int ppb, int lg) {
  extern __shared__ double2 sm[];
  if (ss && halted(ss)) return;
  const int nx = fp.nx, ny = fp.ny;
  const int npairs = nx / 2 + 1;
  const int pair0 = blockIdx.x * ppb;  // ppb column pairs per block
  const int np = min(ppb, npairs - pair0);
  const int nl = 2 * np;
  const int p = fp.p0 + blockIdx.y;
  const int nout = mode == 0 ? 3 : 1;
  const int npts = nl * ny;            // points of one layer
  const int bsz = lg * 2 * ppb * ny;   // points of one buffer
  double2* A = sm;
  double2* B = sm + bsz;
  double2* Z = sm + 2 * bsz;           // used when lg < nout
  // columns of line l: pair (l >> 1), mirror if odd
  for (int q = threadIdx.x; q < npts; q += blockDim.x) {
    const int line = q / ny, y = q - line * ny;
    const int kx = pair0 + (line >> 1);
    const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
    A[line * ny + y] = fp.P[((long long)p * nx + col) * ny + y];
  }
  __syncthreads();
  double2* spec = fft_lines(A, B, ny, fp.logny, nl, fp.twy, false);
  double2* G = (spec == A) ? B : A;  // layer o0 + o's lines at G + o npts
  double2* T = lg == nout ? spec : Z;
  const int nplanes = mode == 0 ? 3 : 1;
  for (int o0 = 0; o0 < nout; o0 += lg) {
  for (int q = threadIdx.x; q < lg * npts; q += blockDim.x) {
    const int o = o0 + q / npts, qq = q - (o - o0) * npts;
    const int line = qq / ny, ky = qq - line * ny;
    const int kx = pair0 + (line >> 1);
    const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
    const double2 F = spec[qq];
    double2 g;
    if (mode == 1) {
      const double kxm = fp.ktx[col], kym = fp.kty[ky];
      const double k2 = kxm * kxm + kym * kym;
      if (k2 > 0.0) {
        const double2 m = make_double2(kxm / k2, kym / k2);
        g = cmul(m, F);
      } else {
        g = make_double2(0.0, 0.0);
      }
    } else if (mode == 4) {
      // F = FFT(v_x + i v_y).  With V_x = (F + conj F(-k)) / 2 and
      // V_y = (F - conj F(-k)) / 2i, the divergence-free part
      // V - k (k . V) / |k|^2 packs as (F - e^(2 i theta) conj F(-k)) / 2,
      // e^(i theta) = (k_x + i k_y) / |k|; times the filter
      // exp(-(2 |k| / k_N)^4).  The mean and the Nyquist modes (whose signed
      // wavenumber has no partner) carry none.
      const double kxw = fp.ktx[col], kyw = fp.kty[ky];
      const double k2 = kxw * kxw + kyw * kyw;
      if (k2 > 0.0 && 2 * col != nx && 2 * ky != ny) {
        const double2 Fm = spec[(line ^ 1) * ny + ((ny - ky) & (ny - 1))];
        const double c2 = (kxw * kxw - kyw * kyw) / k2, s2 = 2.0 * kxw * kyw / k2;
        const double ax = kxw / fp.knx, ay = kyw / fp.kny;
        const double q4 = 4.0 * (ax * ax + ay * ay);
        const double w = 0.5 * exp(-q4 * q4);
        g = make_double2(w * (F.x - (c2 * Fm.x + s2 * Fm.y)), w * (F.y - (s2 * Fm.x - c2 * Fm.y)));
      } else {
        g = make_double2(0.0, 0.0);
      }
    } else if (mode == 2) {
      // transpose of Eq. 7's inversion: with F = FFT(X + i Y) for real X,
      // Y (the adjoints of A_x, A_y), the spectrum of the B_z adjoint is
      // conj(m_x) X + conj(m_y) Y = [(kt_x - i kt_y) F - (kt_x + i kt_y) conj F(-k)] / (2 kt^2)
      const double kxm = fp.ktx[col], kym = fp.kty[ky];
      const double k2 = kxm * kxm + kym * kym;
      if (k2 > 0.0) {
        const double2 Fm = spec[(line ^ 1) * ny + ((ny - ky) & (ny - 1))];
        const double2 Fc = make_double2(Fm.x, -Fm.y);
        const double2 t1 = cmul(make_double2(kxm, -kym), F);
        const double2 t2 = cmul(make_double2(kxm, kym), Fc);
        g = make_double2((t1.x - t2.x) / (2.0 * k2), (t1.y - t2.y) / (2.0 * k2));
      } else {
        g = make_double2(0.0, 0.0);
      }
    } else {
      // ghost layer o + 1: the multipliers of its distance from the top
      // layer (M_t) and, below the photosphere, from the bottom one (M_b)
      const long long e = (long long)o * nx * ny + (long long)col * ny + ky;
      const double mt = fp.et[e], mb = fp.eb[e];
      if (p == 0) {
        g = make_double2(mt * F.x, mt * F.y);
      } else if (p == 1) {
        g = make_double2(mb * F.x, mb * F.y);
      } else {
        const double2 Fm = spec[(line ^ 1) * ny + ((ny - ky) & (ny - 1))];
        const double ca = 0.5 * (mt + mb), cb = 0.5 * (mt - mb);
        g = make_double2(ca * F.x + cb * Fm.x, ca * F.y - cb * Fm.y);
      }
    }
    G[q] = g;
  }
  __syncthreads();
  const double2* r = fft_lines(G, T, ny, fp.logny, lg * nl, fp.twy, true);
  for (int q = threadIdx.x; q < lg * npts; q += blockDim.x) {
    const int o = o0 + q / npts, qq = q - (o - o0) * npts;
    const int line = qq / ny, y = qq - line * ny;
    const int kx = pair0 + (line >> 1);
    const bool self = (kx == 0 || 2 * kx == nx);
    if ((line & 1) && self) continue;  // the mirror of a self-paired column
    const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
    fp.Q[(((long long)o * nplanes + p) * nx + col) * ny + y] = r[q];
  }
  __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 3. inverse rows: normalise by 1/(nx ny); mode 0 writes ghost layers of the
// state, mode 1 the compact planes out_re, out_im ([ny][nx]).
// mode 2 (adjoint): plane c adds its real part into A_c at the top layer and
// its imaginary part into A_c at the photosphere (interior x, y only);
// mode 3: real part into out_re.
template <typename R>
__global__ void __launch_bounds__(256) rows_inv_kernel(FFTPlan fp, Layout L, R* __restrict__ f, R* out_re,
                                                       R* out_im, int mode, const StepState* ss, int nb) {
  extern __shared__ double2 sm[];
  if (ss && halted(ss)) return;
  const int nx = fp.nx, ny = fp.ny;
  const int y0 = blockIdx.x * nb;
  const int p = fp.p0 + blockIdx.y, o = blockIdx.z;
  const int nplanes = mode == 0 ? 3 : (mode == 2 ? 3 : 1);
  double2* a = sm;
  double2* b = sm + nb * nx;
  for (int q = threadIdx.x; q < nb * nx; q += blockDim.x) {
    const int x = q / nb, line = q - x * nb;
    a[line * nx + x] = fp.Q[(((long long)o * nplanes + p) * nx + x) * ny + y0 + line];
  }
  __syncthreads();
  double2* r = fft_lines(a, b, nx, fp.lognx, nb, fp.twx, true);
  const double sc = 1.0 / ((double)nx * (double)ny);
  const int m = o + 1;
  const int ktop = L.nz - 1 + m, kbot = -m;
  for (int q = threadIdx.x; q < nb * nx; q += blockDim.x) {
    const int line = q / nx, x = q - line * nx, y = y0 + line;
    const double2 v = r[line * nx + x];
    const R re = (R)(v.x * sc), im = (R)(v.y * sc);
    if (mode == 1) {
      out_re[(long long)y * nx + x] = re;
      out_im[(long long)y * nx + x] = im;
      continue;
    }
    if (mode == 3) {
      out_re[(long long)y * nx + x] = re;
      continue;
    }
    if (mode == 2) {
      f[L.at(AX + p, L.nz - 1, y, x)] += re;
      f[L.at(AX + p, 0, y, x)] += im;
      continue;
    }
    int f1, k1, f2, k2;
    if (p == 0) { f1 = AX; k1 = ktop; f2 = AY; k2 = ktop; }
    else if (p == 1) { f1 = AX; k1 = kbot; f2 = AY; k2 = kbot; }
    else { f1 = AZ; k1 = ktop; f2 = AZ; k2 = kbot; }
    int xs[3], ys[3], nxs = 1, nys = 1;
    xs[0] = x; ys[0] = y;
    if (x < NG) xs[nxs++] = x + nx;
    if (x >= nx - NG) xs[nxs++] = x - nx;
    if (y < NG) ys[nys++] = y + ny;
    if (y >= ny - NG) ys[nys++] = y - ny;
    for (int bb = 0; bb < nys; ++bb)
      for (int aa = 0; aa < nxs; ++aa) {
        f[L.at(f1, k1, ys[bb], xs[aa])] = re;
        f[L.at(f2, k2, ys[bb], xs[aa])] = im;
      }
  }
}

// Adjoint columns: for component c, sum over the three ghost layers m of the
// extrapolated spectra of the packed ghost adjoints (top real, bottom
// imaginary), then one inverse FFT along y.  Input planes 3c + m - 1 in
// fp.P, output plane c in fp.Q.
__global__ void __launch_bounds__(256) cols_adj_kernel(FFTPlan fp, const StepState* ss, int ppb) {
  extern __shared__ double2 sm[];
  if (ss && halted(ss)) return;
  const int nx = fp.nx, ny = fp.ny;
  const int npairs = nx / 2 + 1;
  const int pair0 = blockIdx.x * ppb;
  const int np = min(ppb, npairs - pair0);
  const int nl = 2 * np;
  const int c = blockIdx.y;
  const int buf = 2 * ppb * ny;
  double2* X = sm;
  double2* Y = sm + buf;
  double2* acc = sm + 2 * buf;
  for (int q = threadIdx.x; q < nl * ny; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
  for (int m = 1; m <= 3; ++m) {
    const int p = 3 * c + m - 1;
    __syncthreads();
    for (int q = threadIdx.x; q < nl * ny; q += blockDim.x) {
      const int line = q / ny, y = q - line * ny;
      const int kx = pair0 + (line >> 1);
      const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
      X[line * ny + y] = fp.P[((long long)p * nx + col) * ny + y];
    }
    __syncthreads();
    double2* spec = fft_lines(X, Y, ny, fp.logny, nl, fp.twy, false);
    for (int q = threadIdx.x; q < nl * ny; q += blockDim.x) {
      const int line = q / ny, ky = q - line * ny;
      const int kx = pair0 + (line >> 1);
      const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
      const long long e = (long long)(m - 1) * nx * ny + (long long)col * ny + ky;
      const double mt = fp.et[e], mb = fp.eb[e];
      const double2 F = spec[line * ny + ky];
      const double2 Fm = spec[(line ^ 1) * ny + ((ny - ky) & (ny - 1))];
      const double ca = 0.5 * (mt + mb), cb = 0.5 * (mt - mb);
      acc[q].x += ca * F.x + cb * Fm.x;
      acc[q].y += ca * F.y - cb * Fm.y;
    }
  }
  __syncthreads();
  double2* r = fft_lines(acc, X, ny, fp.logny, nl, fp.twy, true);
  for (int q = threadIdx.x; q < nl * ny; q += blockDim.x) {
    const int line = q / ny, y = q - line * ny;
    const int kx = pair0 + (line >> 1);
    const bool self = (kx == 0 || 2 * kx == nx);
    if ((line & 1) && self) continue;
    const int col = (line & 1) ? ((nx - kx) & (nx - 1)) : kx;
    fp.Q[((long long)c * nx + col) * ny + y] = r[line * ny + y];
  }
}

// Dynamic shared-memory limits of the FFT kernels, set once per device (the
// attribute belongs to the device's context).
static void set_smem_once() {
  static PerDevice<bool> done;
  done.get([] {
    cudaFuncSetAttribute(rows_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * FFT_PTS * 16);
    cudaFuncSetAttribute(rows_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * FFT_PTS * 16);
    cudaFuncSetAttribute(rows_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * FFT_PTS * 16);
    cudaFuncSetAttribute(rows_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * FFT_PTS * 16);
    cudaFuncSetAttribute(cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 6 * FFT_PTS * 16);
    cudaFuncSetAttribute(cols_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * FFT_PTS * 16);
    return true;
  });
}

// batch sizes: rows per block (nb) so a block holds ~1024 points, column
// pairs per block (ppb) so there are enough blocks for every SM; shared
// memory sized to the batch
struct FFTLaunch {
  int nb, ppb, lg;                          // lg: ghost layers per inverse batch in cols
  size_t smem_rows, smem_cols, smem_cols3;  // cols: one output layer, three
};

static FFTLaunch fft_launch(const FFTPlan& fp) {
  FFTLaunch l;
  l.nb = 1024 / fp.nx;
  if (l.nb < 1) l.nb = 1;
  if (l.nb > fp.ny) l.nb = fp.ny;
  l.ppb = 256 / fp.ny;
  if (l.ppb < 1) l.ppb = 1;
  l.smem_rows = (size_t)2 * l.nb * fp.nx * sizeof(double2);
  l.smem_cols = (size_t)3 * 2 * l.ppb * fp.ny * sizeof(double2);  // also cols_adj_kernel
  // the three ghost layers in one batch while that keeps two column blocks
  // per SM (at most 96 KB), one at a time otherwise (at 1024^2 the batched
  // form, 192 KB and one block per SM, measured 8 % slower)
  l.lg = (size_t)6 * 2 * l.ppb * fp.ny * sizeof(double2) <= (size_t)96 * 1024 ? 3 : 1;
  l.smem_cols3 = (size_t)(l.lg == 3 ? 6 : 3) * 2 * l.ppb * fp.ny * sizeof(double2);
  return l;
}

// Row transforms of `planes` planes: lines per block chosen so that the
// blocks spread evenly over the SMs (all blocks of these kernels are resident
// at once and share each SM's FP64 pipe, so the busiest SM sets the time);
// one thread per radix-4 butterfly of a stage.
struct RowsCfg {
  int nb, threads;
  size_t smem;
};

static RowsCfg rows_cfg(const FFTPlan& fp, int planes) {
  const int nsm = sm_count();
  int nbmax = 1024 / fp.nx;
  if (nbmax < 1) nbmax = 1;
  if (nbmax > fp.ny) nbmax = fp.ny;
  RowsCfg c{nbmax, 0, 0};
  double best = -1.0;
  for (int nb = nbmax; nb >= 1; nb >>= 1) {
    const long long blocks = (long long)planes * (fp.ny / nb);
    const long long per_sm = (blocks + nsm - 1) / nsm;
    const double eff = (double)blocks / (double)(per_sm * nsm);
    if (eff > best + 1e-9) {
      best = eff;
      c.nb = nb;
    }
  }
  c.threads = c.nb * fp.nx / 4;
  if (c.threads > 256) c.threads = 256;
  if (c.threads < 32) c.threads = 32;
  c.smem = (size_t)2 * c.nb * fp.nx * sizeof(double2);
  return c;
}

template <typename R>
void launch_pfe(const FFTPlan& fp, const Layout& L, R* f, const StepState* ss, cudaStream_t st,
                const PlaneStreams* ps) {
  set_smem_once();
  const FFTLaunch l = fft_launch(fp);
  const int npairs = fp.nx / 2 + 1;
  if (!ps) {
    const RowsCfg rf = rows_cfg(fp, 3), ri = rows_cfg(fp, 9);
    rows_fwd_kernel<R><<<dim3(fp.ny / rf.nb, 3), rf.threads, rf.smem, st>>>(fp, L, f, nullptr, 0, ss, rf.nb,
                                                                            nullptr, nullptr);
    cols_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 3), 256, l.smem_cols3, st>>>(fp, 0, ss, l.ppb, l.lg);
    rows_inv_kernel<R><<<dim3(fp.ny / ri.nb, 3, 3), ri.threads, ri.smem, st>>>(fp, L, f, nullptr, nullptr, 0, ss,
                                                                              ri.nb);
    return;
  }
  // one chain (rows, columns, inverse rows) per packed plane, on its own
  // stream: the chains share no data, and running them side by side fills
  // the SMs' FP64 pipes where one launch's tail would leave them idle
  const RowsCfg rf = rows_cfg(fp, 1), ri = rows_cfg(fp, 3);
  cudaEventRecord(ps->fork, st);
  for (int i = 0; i < 2; ++i) cudaStreamWaitEvent(ps->s[i], ps->fork, 0);
  for (int p = 0; p < 3; ++p) {
    cudaStream_t sp = p == 0 ? st : ps->s[p - 1];
    FFTPlan fq = fp;
    fq.p0 = p;
    rows_fwd_kernel<R><<<dim3(fp.ny / rf.nb, 1), rf.threads, rf.smem, sp>>>(fq, L, f, nullptr, 0, ss, rf.nb,
                                                                            nullptr, nullptr);
    cols_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 1), 256, l.smem_cols3, sp>>>(fq, 0, ss, l.ppb, l.lg);
    rows_inv_kernel<R><<<dim3(fp.ny / ri.nb, 1, 3), ri.threads, ri.smem, sp>>>(fq, L, f, nullptr, nullptr, 0, ss,
                                                                              ri.nb);
  }
  for (int i = 0; i < 2; ++i) {
    cudaEventRecord(ps->join[i], ps->s[i]);
    cudaStreamWaitEvent(st, ps->join[i], 0);
  }
}

template <typename R>
void launch_atarget(const FFTPlan& fp, const R* bz, R* axt, R* ayt, cudaStream_t st) {
  set_smem_once();
  Layout L{};
  const FFTLaunch l = fft_launch(fp);
  const int npairs = fp.nx / 2 + 1;
  const RowsCfg r1 = rows_cfg(fp, 1);
  rows_fwd_kernel<R><<<dim3(fp.ny / r1.nb, 1), r1.threads, r1.smem, st>>>(fp, L, nullptr, bz, 1, nullptr, r1.nb,
                                                                          nullptr, nullptr);
  cols_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 1), 256, l.smem_cols, st>>>(fp, 1, nullptr, l.ppb, 1);
  rows_inv_kernel<R><<<dim3(fp.ny / r1.nb, 1, 1), r1.threads, r1.smem, st>>>(fp, L, nullptr, axt, ayt, 1, nullptr,
                                                                             r1.nb);
}

void launch_rotational(const FFTPlan& fp, const double* vx, const double* vy, double* rx, double* ry,
                       cudaStream_t st) {
  set_smem_once();
  Layout L{};
  const FFTLaunch l = fft_launch(fp);
  const int npairs = fp.nx / 2 + 1;
  const RowsCfg r1 = rows_cfg(fp, 1);
  rows_fwd_kernel<double><<<dim3(fp.ny / r1.nb, 1), r1.threads, r1.smem, st>>>(fp, L, nullptr, nullptr, 3, nullptr,
                                                                               r1.nb, vx, vy);
  cols_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 1), 256, l.smem_cols, st>>>(fp, 4, nullptr, l.ppb, 1);
  rows_inv_kernel<double><<<dim3(fp.ny / r1.nb, 1, 1), r1.threads, r1.smem, st>>>(fp, L, nullptr, rx, ry, 1,
                                                                                 nullptr, r1.nb);
}

// Adjoint of the potential-field ghosts: gbar (adjoint of the ghost-filled
// state) has its A ghost-layer entries mapped back onto the top layer and
// the photosphere.  `fp_adj` is the plan with the 9-plane buffer as P and the
// 3-plane buffer as Q.
template <typename R>
void launch_pfe_adjoint(const FFTPlan& fp_adj, const Layout& L, R* gbar, const StepState* ss, cudaStream_t st) {
  set_smem_once();
  const FFTLaunch l = fft_launch(fp_adj);
  const int npairs = fp_adj.nx / 2 + 1;
  const RowsCfg r9 = rows_cfg(fp_adj, 9), r3 = rows_cfg(fp_adj, 3);
  rows_fwd_kernel<R><<<dim3(fp_adj.ny / r9.nb, 9), r9.threads, r9.smem, st>>>(fp_adj, L, gbar, nullptr, 2, ss, r9.nb,
                                                                              nullptr, nullptr);
  cols_adj_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 3), 256, l.smem_cols, st>>>(fp_adj, ss, l.ppb);
  rows_inv_kernel<R><<<dim3(fp_adj.ny / r3.nb, 3, 1), r3.threads, r3.smem, st>>>(fp_adj, L, gbar, nullptr, nullptr, 2,
                                                                                ss, r3.nb);
}

// Transpose of the magnetogram inversion: B_z adjoint (out, [ny][nx]) from
// the FP64 adjoints of A_x, A_y (abx, aby).
template <typename R>
void launch_atarget_adjoint(const FFTPlan& fp, const double* abx, const double* aby, R* out, cudaStream_t st) {
  set_smem_once();
  Layout L{};
  const FFTLaunch l = fft_launch(fp);
  const int npairs = fp.nx / 2 + 1;
  rows_fwd_kernel<R><<<dim3(fp.ny / l.nb, 1), 256, l.smem_rows, st>>>(fp, L, nullptr, nullptr, 3, nullptr, l.nb, abx,
                                                                       aby);
  cols_kernel<<<dim3((npairs + l.ppb - 1) / l.ppb, 1), 256, l.smem_cols, st>>>(fp, 2, nullptr, l.ppb, 1);
  rows_inv_kernel<R><<<dim3(fp.ny / l.nb, 1, 1), 256, l.smem_rows, st>>>(fp, L, nullptr, out, nullptr, 3, nullptr,
                                                                          l.nb);
}

template void launch_pfe_adjoint<float>(const FFTPlan&, const Layout&, float*, const StepState*, cudaStream_t);
template void launch_pfe_adjoint<double>(const FFTPlan&, const Layout&, double*, const StepState*, cudaStream_t);
template void launch_atarget_adjoint<float>(const FFTPlan&, const double*, const double*, float*, cudaStream_t);
template void launch_atarget_adjoint<double>(const FFTPlan&, const double*, const double*, double*, cudaStream_t);
template void launch_pfe<float>(const FFTPlan&, const Layout&, float*, const StepState*, cudaStream_t,
                                const PlaneStreams*);
template void launch_pfe<double>(const FFTPlan&, const Layout&, double*, const StepState*, cudaStream_t,
                                 const PlaneStreams*);
template void launch_atarget<float>(const FFTPlan&, const float*, float*, float*, cudaStream_t);
template void launch_atarget<double>(const FFTPlan&, const double*, double*, double*, cudaStream_t);

}  // namespace mhd
