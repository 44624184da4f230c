// mhd_internal.h -- launchers shared between the translation units of libmhd.
#pragma once
#include <atomic>
#include <climits>
#include <cstdio>
#include <functional>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include "mhd_common.cuh"

namespace mhd {

// Potential-field FFT plan: all arrays live in the caller's workspace.
struct FFTPlan {
  int nx, ny, lognx, logny;
  const double2* twx;  // exp(-2 pi i r / nx), r < nx
  const double2* twy;  // exp(-2 pi i r / ny), r < ny
  const double* et;    // [3][kx][ky] exp(-|k| d_m), ghost layer m above the top (Eq. 17)
  const double* eb;    // [3][kx][ky] exp(+f_b |k| d'_m), ghost layer m below the photosphere (Sect. 2.4)
  const double* ktx;   // modified first-derivative wavenumbers, [nx]
  const double* kty;   // [ny]
  double2* P;          // [3][nx][ny] row spectra, transposed
  double2* Q;          // [3][3][nx][ny] extrapolated spectra, transposed
  int p0;              // first plane of a launch (blockIdx.y offset; 0 unless planes run apart)
  double knx, kny;     // Nyquist wavenumbers pi / dx, pi / dy (the granulation filter only)
};

// three streams for the potential-field planes of one substep: the caller's
// and two more, forked from and joined back to it
struct PlaneStreams {
  cudaStream_t s[2];
  cudaEvent_t fork, join[2];
};

struct Driver {
  const void* axt;  // [ny][nx] A_x of the target magnetogram
  const void* ayt;
  const void* v0;   // [2][ny][nx]
  const void* v1;
};

// set the message returned by mhd_last_error(NULL)
void set_global_error(const char* fmt, ...);

// A value that belongs to a device -- kernel attributes set there, a launch
// geometry from its SM count and occupancy -- computed once per device, under
// a lock: handles on several devices or host threads may launch at once.
template <typename T>
class PerDevice {
 public:
  template <typename F>
  T get(F make) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMax) dev = 0;
    if (ready_[dev].load(std::memory_order_acquire)) return val_[dev];
    std::lock_guard<std::mutex> lock(mu_);
    if (!ready_[dev].load(std::memory_order_relaxed)) {
      val_[dev] = make();
      ready_[dev].store(true, std::memory_order_release);
    }
    return val_[dev];
  }

 private:
  static constexpr int kMax = 64;
  std::mutex mu_;
  std::atomic<bool> ready_[kMax]{};
  T val_[kMax]{};
};

// SM count of the current device
inline int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  return n;
}

constexpr int FFT_PTS = 2048;          // complex points per shared buffer
constexpr int RED_BLOCKS_MAX = 4096;   // partial-reduction slots
constexpr int CFL_SLOTS = 256;         // CFL maxima slot pairs (after the partials)

// ghost fill
template <typename R> void launch_rims(const Layout& L, R* f, int k0, int k1, cudaStream_t st);
template <typename R> void launch_init_u_ghosts(const Layout& L, R* f, cudaStream_t st);
template <typename R> void launch_bc(const Layout& L, const Phys<R>& ph, const Background<R>& bg, R* f,
                                     R dz, const StepState* ss, cudaStream_t st);
// potential-field ghosts of A (three FFT kernels)
// (ps: run the three planes on three streams; nullptr: one stream)
template <typename R> void launch_pfe(const FFTPlan& fp, const Layout& L, R* f, const StepState* ss,
                                      cudaStream_t st, const PlaneStreams* ps = nullptr);
// vector potential of the target magnetogram into axt, ayt
template <typename R> void launch_atarget(const FFTPlan& fp, const R* bz, R* axt, R* ayt, cudaStream_t st);
// filtered rotational part (Eq. 3) of the plane field (vx, vy) into (rx, ry),
// all [ny][nx]; fp.ktx, fp.kty hold the signed wavenumbers 2 pi m / L
void launch_rotational(const FFTPlan& fp, const double* vx, const double* vy, double* rx, double* ry,
                       cudaStream_t st);
// fused right-hand side + RK update; sub = 0,1,2, or -1 to write the raw RHS into df
template <typename R> void launch_rk(const Layout& L, const Phys<R>& ph, const Background<R>& bg,
                                     const R* fin, R* fout, R* df,
                                     const R* wtab, const R* wptab, const Driver& drv, const StepState* ss,
                                     int sub, cudaStream_t st);
// FP32 TMA-fed variant of launch_rk (tensor map of the input state set)
void launch_rk_tiled(const CUtensorMap* tm, const Layout& L, const Phys<float>& ph, const Background<float>& bg,
                     float* fout, float* df, const float* wtab, const float* wptab, const Driver& drv,
                     StepState* ss, int sub, double dx, double dy, double dz, cudaStream_t st);
// FP32 pointwise adjoint of substep `sub` on the TMA-fed z-march (tm maps the
// ghost-filled substep state): 46 coefficient fields and the driver adjoints
void launch_adj_point_tiled(const CUtensorMap* tm, const Layout& L, const Phys<float>& ph,
                            const Background<float>& bg, const float* dbar, float* coef, double* thbar,
                            const float* wtab, const float* wptab, StepState* ss, int sub, double dx, double dy,
                            double dz, cudaStream_t st);
// tensor map of one padded FP32 state set (dims mx, my, mz, 8 fields) whose box is
// one plane (box_x x box_y x 1; default a 32 x 8 tile with its halo, 40 x 14)
// of box_fields consecutive fields
int make_state_tensor_map(CUtensorMap* tm, const Layout& L, void* base, int box_fields = NF, int box_x = 40,
                          int box_y = 14);
// FP32 right-hand side + RK update as two z-march passes (A -> B, J, swamp terms;
// then u, ln rho, ln T with the physics and the update); tm_a, tm_r map the input
// state with 3-field (A) and 5-field (u_x .. ln T) boxes
void launch_rk_split(const CUtensorMap* tm_a, const CUtensorMap* tm_r, const Layout& L, const Phys<float>& ph,
                     const Background<float>& bg, const float* fin, float* fout, float* df, float* bj, float* sw,
                     int ksw, const float* wtab, const float* wptab, const Driver& drv, StepState* ss, int sub,
                     double dx, double dy, double dz, cudaStream_t st);
// FP32 right-hand side + RK update in one z-march pass, two x-adjacent cells
// per thread (f32x2), z histories in TMEM; tm maps the input state with
// 8-field halo boxes, tmd the RK accumulator with 8-field 32 x 8 tiles.
// Requires nx even, nx >= 8, ny >= 6.
bool rk_pair_supported(const Layout& L);
// skip_plane, wait_limit: the time-out test hook (mhd_debug_skip_copy); INT_MIN
// for a normal launch
void launch_rk_pair(const CUtensorMap* tm, const CUtensorMap* tmd, const Layout& L, const Phys<float>& ph, const Background<float>& bg,
                    float* fout, float* df, const float* wtab, const float* wptab, const Driver& drv, StepState* ss,
                    int sub, double dx, double dy, double dz, cudaStream_t st, int skip_plane = INT_MIN,
                    int wait_limit = 0);
// pointwise adjoint of substep sub on the same z-march (tm: the ghost-filled
// substep state, tmd: D, the adjoint of the RK accumulator, 32 x 8 tiles)
void launch_adj_point_pair(const CUtensorMap* tm, const CUtensorMap* tmd, const Layout& L, const Phys<float>& ph,
                           const Background<float>& bg, const float* dbar, float* coef, double* thbar,
                           const float* wtab, const float* wptab, StepState* ss, int sub, double dx, double dy,
                           double dz, cudaStream_t st);
// adjoint (transposed linearisation of one substep)
constexpr int NCOEF_ADJ = 40;
template <typename R> void launch_adj_point(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* g,
                                            const R* dbar, R* coef, double* thbar, const R* wtab, const R* wptab,
                                            const StepState* ss, int sub, cudaStream_t st);
template <typename R> void launch_adj_gather(const Layout& L, const Phys<R>& ph, const R* coef, const R* dbar,
                                             R* gbar, const StepState* ss, cudaStream_t st);
// tiled gather (needs adj_gather_tiled_ok): folds the in-plane grad-div terms into the
// coefficients first (coef is modified); on layers klo <= k < khi it also applies the
// substep's update F += G, D = alpha D + beta F, elsewhere it stores G in gbar
bool adj_gather_tiled_ok(const Layout& L);
template <typename R> void launch_adj_gather_tiled(const Layout& L, const Phys<R>& ph, R* coef, R* dbar, R* gbar,
                                                   R* fbar, double alpha, double beta, int klo, int khi,
                                                   const StepState* ss, cudaStream_t st);
// the same contract as a z-march over coefficient planes (coef is not modified): a
// CTA stages one output group's 20 coefficient fields plane by plane and
// scatters the z stencils into a register ring (needs adj_gather_tiled_ok)
template <typename R> void launch_adj_gather_zm(const Layout& L, const Phys<R>& ph, const R* coef, R* dbar, R* gbar,
                                                R* fbar, double alpha, double beta, int klo, int khi, StepState* ss,
                                                cudaStream_t st);
template <typename R> void launch_adj_bc(const Layout& L, const Phys<R>& ph, const Background<R>& bg, const R* g,
                                         R* gbar, R dz, const StepState* ss, cudaStream_t st);
// adjoint elementwise updates (mode 0: D = beta F; mode 1: F += G, D = alpha D + beta F),
// skipping interior layers klo <= k < khi; nx must be a multiple of 4 and
// NF * (nz + 6) * ny * nx / 4 < 2^31
template <typename R> void launch_adj_update(const Layout& L, R* fbar, R* dbar, const R* gbar, double alpha,
                                             double beta, int mode, int klo, int khi, const StepState* ss,
                                             cudaStream_t st);
template <typename R> void launch_bz_plane(int nx, int ny, int nz, int k, double dx, double dy, const R* st_in,
                                           R* out, int adjoint, const R* bbar, R* lam, cudaStream_t st);
template <typename R> void launch_adj_pack(const Layout& L, int bcz, const R* fbar, R* out, cudaStream_t st);
template <typename R> void launch_adj_unpack(const Layout& L, const R* in, R* fbar, cudaStream_t st);
template <typename R> void launch_d2r(const double* in, R* out, long long n, cudaStream_t st);
template <typename R> void launch_pfe_adjoint(const FFTPlan& fp_adj, const Layout& L, R* gbar, const StepState* ss,
                                              cudaStream_t st);
template <typename R> void launch_atarget_adjoint(const FFTPlan& fp, const double* abx, const double* aby, R* out,
                                                  cudaStream_t st);
// A stored about a fixed background (params a_background): FP64 packed
// [3][nz][ny][nx] into fields 0..2 of a padded FP64 array (interior and x,y
// images); a perturbation A' into the state's fields 0..2 likewise; periodic
// z ghosts of the FP64 background (bc_z = 1); the per-cell tables B, J and the
// swamp-layer lap A, div A of the ghost-filled background, its photospheric
// A_x, A_y (FP64, a0 [2][ny][nx]) and its padded copy in the state precision
// (abg, 3 fields); the nudging target relative to the background,
// rel = at - a0 over n values; R -> FP64 widening
void launch_abg_unpack64(const Layout& L, const double* in, double* a, cudaStream_t st);
template <typename R> void launch_abg_pert(const Layout& L, const R* in, R* f, cudaStream_t st);
void launch_abg_zper(const Layout& L, double* a, cudaStream_t st);
template <typename R> void launch_abg_tables(const Layout& L, double dx, double dy, double dz, const double* zm,
                                             const double* a, R* bB, R* bJ, R* bL, int ksw, double* a0, R* abg,
                                             cudaStream_t st);
template <typename R> void launch_abg_target(const double* at, const double* a0, R* rel, long long n,
                                             cudaStream_t st);
template <typename R> void launch_widen(const R* in, double* out, long long n, cudaStream_t st);
// throughput probe: `iters` rounds of 8 independent FMA chains per thread
// over grid x 256 threads, in R (instrumentation, not a step of the method)
template <typename R> void launch_fma_probe(R* out, int grid, int iters, cudaStream_t st);

// Snapshot files in the paper's HDF5 layout (mhd_h5.cu): var.h5 (time,
// data/<variable> with outer ghosts, grid, settings) and grid.h5; either path
// may be null.  field(f, fp) writes field f's [nz+6][ny+6][nx+6] values in
// the handle's precision to fp.  0, or -1 on an I/O error.
}  // namespace mhd
struct mhd_params;
namespace mhd {
int h5_write_snapshot(const char* var_path, const char* grid_path, const mhd_params* p, double t,
                      const std::function<bool(int, FILE*)>& field);
// reductions
// CFL block maxima by atomicMax into CFL_SLOTS slot pairs at `partial`
// (zeroed first when `zero`); the planes: all, the inner ones whose stencils
// read no ghost plane (k = 3 .. nz - 4), or the three at each end.  Returns
// the slot count for launch_cfl_finalize.
enum class CflPlanes { all, inner, ends };
template <typename R> int launch_cfl_partial(const Layout& L, const Phys<R>& ph, const Background<R>& bg,
                                             const R* f, const R* wtab, double* partial, StepState* ss,
                                             CflPlanes planes, bool zero, cudaStream_t st);
// the same maxima over the inner layers for the FP32 state as a TMA-fed
// z-march (mhd_cfl_zm.cu); tma: the state set's boxes of A (40 x 14 x 3)
int launch_cfl_inner_zm(const CUtensorMap* tma, const Layout& L, const Phys<float>& ph, const Background<float>& bg,
                        const float* f, const float* wtab, double* partial, StepState* ss, bool zero,
                        cudaStream_t st);
void launch_cfl_finalize(const double* partial, int nblk, StepState* ss, double c_adv, double c_diff,
                         double dt_fixed, double inv2sum, double t0, double t1, double t_ramp, int probe,
                         cudaStream_t st);
// diagnostics partials; bsc = three scratch fields in the state layout
// (overwritten), e.g. the RK accumulator between steps
template <typename R> int launch_stats_partial(const Layout& L, const Phys<R>& ph, const Background<R>& bg,
                                               const R* f, R* bsc, double* partial, cudaStream_t st);
void launch_stats_finalize(const double* partial, int nblk, StepState* ss, double dv, double da, double gm1,
                           cudaStream_t st);
// pack / unpack interior <-> padded
// (the background is added on the way out and removed on the way in)
template <typename R> void launch_pack(const Layout& L, const Background<R>& bg, const R* f, R* out, int field,
                                       cudaStream_t st);
template <typename R> void launch_unpack(const Layout& L, const Background<R>& bg, const R* in, R* f,
                                         cudaStream_t st);
// padded copy with the background added (diagnostics)
template <typename R> void launch_pack_padded(const Layout& L, const Background<R>& bg, const R* f, R* out,
                                              cudaStream_t st);
// one layer k (0 .. nz-1) of one field into out [ny][nx], background added
template <typename R> void launch_pack_plane(const Layout& L, const Background<R>& bg, const R* f, R* out, int field,
                                             int k, cudaStream_t st);
// per-layer FP64 mean of field `field` of an interior-packed state
template <typename R> void launch_layer_mean(const Layout& L, const R* in, int field, double* out,
                                             cudaStream_t st);

}  // namespace mhd
