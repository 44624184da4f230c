// mhd_static.cu -- allocation-free variant of the magnetogram inversion
// (the vector potential A_x, A_y of a B_z plane computed by mhd_set_driver).
//
// Some callers cannot allocate device memory: a host application that
// reserves the whole GPU up front and hands out no further memory, a plugin
// loaded into a process whose caching allocator already holds nearly all of
// HBM (so a cudaMalloc would fail, or force the framework to release cached
// blocks with a device-wide synchronisation), or code on a latency-critical
// path that must not pay for an allocation.  This entry point needs no
// workspace: its FFT scratch (two complex FP64 planes, twiddles and modified
// wavenumbers) lives in one file-scope __device__ array of fixed size.  The
// array belongs to this file's device module: under CUDA's default lazy
// module loading the module, and with it the array, is loaded on a device by
// the first call there, and stays until the process exits or the context is
// destroyed.
#include <cuda.h>

#include <mutex>

#include "../../include/mhd.h"
#include "mhd_internal.h"

namespace {
constexpr int kStaticMaxN = 512;  // nx, ny <= 512
constexpr size_t kN2 = (size_t)kStaticMaxN * kStaticMaxN;
constexpr size_t kOffP = 0;                                  // double2 [nx * ny]
constexpr size_t kOffQ = kOffP + kN2 * 16;                   // double2 [nx * ny]
constexpr size_t kOffTwx = kOffQ + kN2 * 16;                 // double2 [nx]
constexpr size_t kOffTwy = kOffTwx + (size_t)kStaticMaxN * 16;  // double2 [ny]
constexpr size_t kOffKtx = kOffTwy + (size_t)kStaticMaxN * 16;  // double [nx]
constexpr size_t kOffKty = kOffKtx + (size_t)kStaticMaxN * 8;   // double [ny]
constexpr size_t kStaticBytes = kOffKty + (size_t)kStaticMaxN * 8;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
// Device address of the array per device, and the id of the context it was
// looked up in: a context destroyed and created again (cudaDeviceReset)
// reloads the module at another address, so the id is checked on every call.
void* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points,
// so that the library does not link libcuda itself (it must load on hosts
// without a driver for the ABI checks).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {  // called with g_mu held
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return false;
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

// 8.0 MiB + 24 KiB of FFT scratch, shared by every call on a device.
static __device__ __align__(256) unsigned char g_inv_scratch[kStaticBytes];

namespace mhd {

// Twiddles exp(-2 pi i r / n) and the modified wavenumber of the sixth-order
// first derivative (zero at m = 0 and at the Nyquist mode), written into the
// scratch array.  Every table entry a call reads is rewritten by that call.
__global__ void static_tables_kernel(unsigned char* base, int nx, int ny, double dx, double dy) {
  double2* twx = (double2*)(base + kOffTwx);
  double2* twy = (double2*)(base + kOffTwy);
  double* ktx = (double*)(base + kOffKtx);
  double* kty = (double*)(base + kOffKty);
  const int nmax = nx > ny ? nx : ny;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nmax; r += gridDim.x * blockDim.x) {
    for (int axis = 0; axis < 2; ++axis) {
      const int n = axis == 0 ? nx : ny;
      if (r >= n) continue;
      double s, c;
      sincospi(2.0 * (double)r / (double)n, &s, &c);
      (axis == 0 ? twx : twy)[r] = make_double2(c, -s);
      double kt = 0.0;
      if (r != 0 && 2 * r != n) {
        const double a = 2.0 * (double)(2 * r > n ? r - n : r) / (double)n;  // theta / pi
        kt = (45.0 * sinpi(a) - 9.0 * sinpi(2.0 * a) + sinpi(3.0 * a)) / (30.0 * (axis == 0 ? dx : dy));
      }
      (axis == 0 ? ktx : kty)[r] = kt;
    }
  }
}

}  // namespace mhd

using namespace mhd;

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

extern "C" int mhd_invert_magnetogram_static(int nx, int ny, double dx, double dy, int precision,
                                             const void* bz, void* ax, void* ay, void* stream) {
  if (precision != 32 && precision != 64) {
    set_global_error("mhd_invert_magnetogram_static: precision must be 32 or 64");
    return MHD_ERR_ARG;
  }
  if (!pow2_in(nx, 8, kStaticMaxN) || !pow2_in(ny, 8, kStaticMaxN)) {
    set_global_error("mhd_invert_magnetogram_static: nx = %d, ny = %d; both must be powers of two in [8, %d] "
                     "(the static scratch holds at most %d x %d points)",
                     nx, ny, kStaticMaxN, kStaticMaxN, kStaticMaxN);
    return MHD_ERR_ARG;
  }
  if (!(dx > 0.0) || !(dy > 0.0)) {
    set_global_error("mhd_invert_magnetogram_static: dx, dy must be positive");
    return MHD_ERR_ARG;
  }
  if (!bz || !ax || !ay) {
    set_global_error("mhd_invert_magnetogram_static: bz, ax, ay must be device pointers");
    return MHD_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error("mhd_invert_magnetogram_static: no usable current device (%s)", cudaGetErrorString(e));
    return MHD_ERR_CUDA;
  }
  unsigned char* base;
  {
    // once per device (and again after its context was recreated), with that
    // device current: the device address of the array (its host-side name is
    // only a stand-in).  The lookup also makes the device's primary context
    // current when the calling thread has none yet.
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx);
    if (!have_ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_inv_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error("mhd_invert_magnetogram_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return MHD_ERR_CUDA;
      }
      if (!have_ctx && !current_context_id(&ctx)) {
        set_global_error("mhd_invert_magnetogram_static: no current CUDA context after the symbol lookup");
        return MHD_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = ctx;
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  FFTPlan fp;
  fp.p0 = 0;
  fp.nx = nx;
  fp.ny = ny;
  fp.lognx = 0;
  while ((1 << fp.lognx) < nx) ++fp.lognx;
  fp.logny = 0;
  while ((1 << fp.logny) < ny) ++fp.logny;
  fp.twx = (const double2*)(base + kOffTwx);
  fp.twy = (const double2*)(base + kOffTwy);
  fp.et = nullptr;
  fp.eb = nullptr;
  fp.ktx = (const double*)(base + kOffKtx);
  fp.kty = (const double*)(base + kOffKty);
  fp.P = (double2*)(base + kOffP);
  fp.Q = (double2*)(base + kOffQ);
  // P and Q are fully overwritten by the transform before they are read, so
  // nothing left by an earlier call has to be cleared.
  static_tables_kernel<<<4, 256, 0, st>>>(base, nx, ny, dx, dy);
  if (precision == 64)
    launch_atarget<double>(fp, (const double*)bz, (double*)ax, (double*)ay, st);
  else
    launch_atarget<float>(fp, (const float*)bz, (float*)ax, (float*)ay, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error("mhd_invert_magnetogram_static: launch failed: %s", cudaGetErrorString(e));
    return MHD_ERR_CUDA;
  }
  return MHD_OK;
}
