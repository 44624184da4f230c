/*
 * mhd.h -- C ABI of the GB300 driven coronal MHD library (libmhd.so).
 *
 * One low-storage third-order Runge-Kutta step of compressible resistive MHD
 * in vector-potential form with state (A, u, ln rho, ln T), sixth-order
 * centred differences, and the boundary conditions of Bourdin (2019),
 * "Driving solar coronal MHD simulations on high-performance computers":
 * photospheric nudging toward a magnetogram and a driver velocity
 * (Sect. 2.1, 2.3, Eq. 5), inverted potential-field extrapolation below the
 * photosphere (Sect. 2.4), hydrostatic / symmetric atmospheric ghosts
 * (Sect. 2.5 Eq. 8, Sect. 4.1 Eqs. 11, 13), regular potential-field
 * extrapolation above the top (Sect. 4.2, Eqs. 16-17) and the swamp layer
 * (Sect. 4.3, Eqs. 18-20); its adjoint; and a generator of granulation
 * driver velocities (Sect. 2.3, Eqs. 1-4, the mhd_gran_* calls).
 *
 * Conventions shared by every entry point
 * - Fields, in this order: Ax, Ay, Az, ux, uy, uz, ln rho, ln T (the
 *   variables the paper's snapshots hold, Sect. 5.3).
 * - State arrays are interior-only, C order with x fastest:
 *   [field][z][y][x] = [8][nz][ny][nx]; 2D arrays are [ny][nx]; driver
 *   velocities are [2][ny][nx] (vx, vy).  z index 0 is the photosphere.
 * - Element type = the handle's precision (float for 32, double for 64).
 * - `mem` selects where a caller array lives: MHD_MEM_DEVICE (device pointer,
 *   copied device-to-device on the handle's stream) or MHD_MEM_HOST (host
 *   pointer; the call copies and returns when the host buffer may be reused).
 * - The library never allocates device memory: the caller passes one
 *   workspace of mhd_workspace_bytes() bytes (256-byte aligned) and owns it;
 *   mhd_destroy() frees only host-side bookkeeping.
 * - Every launch is ordered on the stream given to mhd_create(); calls are
 *   asynchronous unless stated otherwise.  With the potential-field boundary,
 *   the FFT of each step's first substep runs on a library-owned
 *   highest-priority stream, and the FFTs of the three packed boundary
 *   planes run side by side on it and two more such streams; all are forked
 *   from and joined back to that stream by events (created by mhd_create,
 *   released by mhd_destroy), so the caller's stream still orders all of the
 *   handle's work.
 * - Return value: MHD_OK (0) or a negative MHD_ERR_* code; the message is
 *   available from mhd_last_error().  Argument errors are reported before any
 *   launch.  A non-finite value met by the time-step reduction (or a device
 *   wait that exceeded its bound) sets a device flag: from then on every
 *   kernel of the handle returns without work, and the next synchronising
 *   call returns MHD_ERR_NONFINITE (or MHD_ERR_TIMEOUT).
 */
#ifndef MHD_H
#define MHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MHD_OK 0
#define MHD_ERR_ARG (-1)        /* invalid argument, shape or pointer        */
#define MHD_ERR_WORKSPACE (-2)  /* workspace missing, misaligned or too small */
#define MHD_ERR_CUDA (-3)       /* a CUDA runtime call failed                 */
#define MHD_ERR_NONFINITE (-4)  /* NaN/Inf detected in the state              */
#define MHD_ERR_UNSUPPORTED (-5)/* valid but not built (e.g. FFT size)        */
#define MHD_ERR_TIMEOUT (-6)    /* a bounded device wait gave up              */
#define MHD_ERR_IO (-7)         /* a snapshot file could not be written       */

#define MHD_MEM_DEVICE 0
#define MHD_MEM_HOST 1

#define MHD_NFIELD 8
#define MHD_NGHOST 3

/* Scheme parameters, code units (mu0 = 1, p = rho T).  Geometry: interior
 * nx x ny x nz cells, periodic in x and y; nx, ny powers of two in [8, 1024]
 * when bc_z = 0 (the potential-field boundary needs the FFT), any size >= 4
 * otherwise; nz >= 7. */
typedef struct mhd_params {
  int nx, ny, nz;
  int precision;       /* 32 or 64: state storage and stencil arithmetic */
  int bc_z;            /* 0: the paper's boundaries; 1: periodic in z (tests) */
  int stats_every;     /* compute diagnostics every n steps (0: never) */
  int adjoint;         /* 1: also reserve the buffers of mhd_adjoint_step (needs
                          8 (nz + 6) ny nx / 4 < 2^31) */
  double dx, dy, dz;
  double gamma;        /* ratio of specific heats */
  double gz;           /* gravity, signed (< 0 points down) */
  double nu;           /* kinematic viscosity */
  double eta;          /* magnetic diffusivity */
  double kappa0;       /* Spitzer coefficient, kappa = kappa0 T^{5/2} */
  double diff_rho;     /* mass diffusivity D_rho (Sect. 2.5) */
  double eta_swamp;    /* swamp magnetic diffusivity eta_s (Eq. 18) */
  double chi_swamp;    /* swamp heat diffusivity chi_s on ln T (Eq. 19) */
  double diffrho_swamp;/* swamp mass diffusivity chi_rho on ln rho (Eq. 20) */
  double z_swamp_start, z_swamp_end; /* cubic weight from 0 to 1 (Sect. 4.3) */
  double tau_u;        /* velocity nudging rate (Eq. 5) */
  double tau_A;        /* magnetic nudging rate at the photosphere (Sect. 2.1) */
  double t_ramp;       /* linear driver switch-on time (Sect. 2.3); <= 0: off */
  double f_pfe_bottom; /* contrast-growth factor of the inverted extrapolation (0.2) */
  double c_adv, c_diff;/* CFL coefficients */
  double dt_fixed;     /* > 0: fixed time step instead of the CFL rule */
  double bext[3];      /* uniform external field added to curl A */
  /* Newtonian cooling of the chromosphere (Sect. 3.1, Eqs. 9-10), read as a
   * relaxation d ln T/dt += -nc_tau (1 - T* / T) c_rho c_z with
   * T* = sqrt(T0(z) T'(rho)), T'(rho) = T0(z') where ln rho0(z') = ln rho
   * (piecewise-linear inverse of the initial profile over the layers, clamped
   * at its ends).  c_rho: 1 down to nc_lnrho_magn - nc_lnrho_width e-folds
   * below the photospheric density, a cosine step to 0 at nc_lnrho_magn;
   * c_z: 1 up to nc_z_max - nc_z_width, a cosine step to 0 at nc_z_max.
   * nc_tau = 0 turns the term off; with nc_tau > 0 the initial ln rho profile
   * must fall strictly with height. */
  double nc_tau;       /* inverse relaxation time (the paper: 0.5 / s) */
  double nc_lnrho_magn, nc_lnrho_width; /* density cut-off: 8 and 2 e-folds */
  double nc_z_max, nc_z_width;          /* height cut-off (3 and 0.3 Mm) */
  /* 1: store A as a perturbation A' = A - A_bg about a fixed background field
   * A_bg given in FP64 by mhd_set_a_background (zero until then), the way ln
   * rho and ln T are stored about their profiles.  The workspace then also
   * holds, per interior cell, the background's B_bg = curl A_bg and
   * J_bg = grad div A_bg - lap A_bg (FP64 stencils, stored in the state
   * precision), lap A_bg and div A_bg on the swamp layers, and A_bg itself.
   * The discrete equations are unchanged (the stencils are linear); FP32
   * rounding then scales with |A'| instead of |A|, which matters where A is
   * large (hundreds in the production-size box).  Not with adjoint = 1. */
  int a_background;
  /* Non-uniform vertical grid (Sect. 1: the spacing grows from about 100 km
   * in the photosphere to about 800 km in the corona; the snapshots carry
   * the inverse spacing dz_1, Sect. 5.3): NULL for z_k = k dz, or a host
   * array of the nz + 6 strictly increasing positions of the layers
   * k = -3 .. nz + 2, read by mhd_workspace_bytes and mhd_create only.  The
   * layer index is the uniform coordinate: dz/dxi and d2z/dxi2 come from the
   * same sixth-order stencils, every z derivative follows by the chain rule,
   * the ghost rules (Eqs. 8, 13) and the potential-field extrapolations
   * (Eq. 17 and its inverted form) take the layer distances, the CFL rule the
   * local spacing, the diagnostics the cell extents (z_{k+1} - z_{k-1}) / 2,
   * the swamp weight and the cooling cut-off the positions.  dz is then
   * unused.  Needs the default FP32 kernel or MHD_RK_VARIANT=simple; not
   * with adjoint = 1. */
  const double* z;
} mhd_params;

/* Diagnostics of the ghost-filled state at time t (FP64 sums). */
typedef struct mhd_stats {
  double t, dt;        /* time of the state; last time step taken */
  double e_kin;        /* sum rho u^2 / 2 dV */
  double e_mag;        /* sum B^2 / 2 dV */
  double e_th;         /* sum rho T / (gamma - 1) dV */
  double mass;         /* sum rho dV */
  double flux_net;     /* sum B_z(z = 0) dx dy (flux balance, Sect. 2.1) */
  double flux_abs;     /* sum |B_z(z = 0)| dx dy */
  double divb_max;     /* max |div B| (zero for B = curl A, Eq. 6) */
  long long step;      /* number of RK steps taken */
  int nonfinite;       /* nonzero once a NaN/Inf was met */
  int pad_;
} mhd_stats;

typedef struct mhd_ctx* mhd_handle;

/* Bytes of device workspace a handle with these parameters needs
 * (0 if the parameters are invalid). */
size_t mhd_workspace_bytes(const mhd_params* p);

/* Create a handle.  workspace: caller-owned device memory of at least
 * mhd_workspace_bytes(p) bytes, 256-byte aligned, kept alive until
 * mhd_destroy.  init_state: [8][nz][ny][nx] initial state (mem selects host or
 * device).  lnrho0: host array of nz + 6 doubles, the initial ln rho profile
 * rho0(z) at z indices -3 .. nz+2; the three values below the photosphere are
 * the fixed density ghosts (Sect. 2.5, 'fg').  lnT0: host array of nz + 6
 * doubles, the initial ln T stratification T0(z) (Sect. 3.1), or NULL to use
 * the layer means of init_state.  ln rho and ln T are stored as perturbations
 * about these FP64 profiles (the equations are unchanged; FP32 rounding then
 * scales with the perturbation).  The stateful horizontal-velocity ghost
 * layers below the photosphere (Eq. 5 acts on j in {0,-1,-2,-3}) start equal
 * to the photospheric layer.  stream: a cudaStream_t (NULL: the legacy default
 * stream).  Synchronises the stream before returning. */
int mhd_create(const mhd_params* p, void* workspace, size_t ws_bytes,
               const void* init_state, int mem, const double* lnrho0,
               const double* lnT0, void* stream, mhd_handle* out);

/* Set the photospheric driver (Sect. 2.1, 2.3): the target magnetogram
 * bz [ny][nx] (flux balanced by the caller) and two velocity snapshots
 * v0, v1 [2][ny][nx] taken at times t0 < t1, interpolated linearly in time and
 * multiplied by the switch-on ramp.  The vector potential of bz (Eq. 7, Weyl
 * gauge, A_z = 0) is computed here with the FP64 FFT.  Must be called before
 * the first mhd_step. */
int mhd_set_driver(mhd_handle h, const void* bz, const void* v0,
                   const void* v1, double t0, double t1, int mem);

/* Advance the state by nsteps full RK3 steps (three substeps each: ghost
 * fill, potential-field FFT, fused right-hand side + RK update; the time step
 * from the FP64 CFL reduction at the first substep).  Asynchronous; no host
 * synchronisation, so the calls may be captured into a CUDA graph on the
 * handle's stream.  Each substep swaps the two state sets on the host: a
 * graph replays correctly when it holds an even number of steps, and the
 * diagnostics schedule (stats_every) is the one seen at capture. */
int mhd_step(mhd_handle h, int nsteps);

/* Background of the vector potential (needs params.a_background = 1; not a
 * step of the paper's method but a storage format, like the ln rho and ln T
 * profiles of mhd_create).  Sets A = a_bg + a_pert, stored as the fixed
 * background a_bg and the perturbation A' = a_pert:
 *   a_bg: [3][nz][ny][nx] FP64 (A_x, A_y, A_z; mem selects host or device),
 *     typically the initial potential field in FP64.  Its ghost layers come
 *     from the same boundary rules as the state's (the potential-field
 *     extrapolations of Sect. 4.2 and 2.4, or periodic copies when bc_z = 1),
 *     applied once here in FP64.
 *   a_pert: [3][nz][ny][nx] in the handle's precision (same mem), or NULL
 *     for A' = 0.
 * The other five fields are left as they are.  Afterwards mhd_read and
 * mhd_read_padded return A' + A_bg (A_bg rounded to the handle's precision),
 * mhd_write stores A' = A - A_bg, and the diagnostics, the CFL rule and the
 * nudging of A_hor toward the target (whose difference from A_bg at the
 * photosphere is formed in FP64) see the full A; max |div B| is that of
 * curl A' (div curl A_bg vanishes to FP64 rounding).  May be called again
 * (each call replaces the background and the state's A).  Synchronises the
 * stream. */
int mhd_set_a_background(mhd_handle h, const double* a_bg, const void* a_pert, int mem);

/* Copy layer k (0 .. nz-1) of one field (0..7) into dst ([ny][nx]); the
 * same values mhd_read returns for that layer.  With MHD_MEM_HOST the call
 * synchronises the stream. */
int mhd_read_plane(mhd_handle h, int field, int k, void* dst, int mem);

/* Arithmetic throughput of the current device in the given precision (32 or
 * 64): eight independent fused multiply-add chains per thread, 8 blocks of
 * 256 threads per SM, timed with CUDA events on `stream` (the best of three
 * launches after one warm-up), written to *flops_per_s (2 flops per FMA).
 * scratch: any device pointer to at least 8 x SM-count elements (written
 * only in a case that does not occur).  Instrumentation for the rooflines
 * of the ALU-bound kernels; synchronises the stream; errors through
 * mhd_last_error(NULL). */
int mhd_fma_peak(int precision, void* scratch, void* stream, double* flops_per_s);

/* Test hook of the bounded device waits (not part of the method): the next
 * launch of the FP32 fused kernel (the default FP32 path) skips, in the
 * first work item of its first CTA, the copy of state plane `plane`
 * (-3 .. nz + 2, of that item's z chunk) together with its barrier arrival,
 * so the wait for that plane finds no copy in flight and gives up after
 * `wait_limit` polls; every wait of that launch uses this limit.  The CTA
 * then drains its copies in flight, frees its tensor memory, records the
 * time-out in the device flag and returns; the step is left incomplete, the
 * following kernels of the handle return without work, and the next
 * synchronising call returns MHD_ERR_TIMEOUT.  mhd_write clears the flag.
 * MHD_ERR_UNSUPPORTED for an FP64 handle or another FP32 kernel variant. */
int mhd_debug_skip_copy(mhd_handle h, int plane, int wait_limit);

/* Copy the interior of one field (0..7) or of all fields (-1) into dst
 * ([nz][ny][nx] or [8][nz][ny][nx]).  With MHD_MEM_HOST the call
 * synchronises the stream. */
int mhd_read(mhd_handle h, int field, void* dst, int mem);

/* Copy the whole state into the handle (same layout as init_state); the
 * stateful velocity ghosts are reset to the photospheric layer.  Also clears
 * the device flag of a non-finite value or a timed-out wait, so a handle
 * halted by either can be stepped again from the state written. */
int mhd_write(mhd_handle h, const void* src, int mem);

/* Synchronise the stream and return the diagnostics of the last step that
 * computed them (stats_every), plus time, dt and step count. */
int mhd_read_stats(mhd_handle h, mhd_stats* out);

/* Set the time of the current state (e.g. to restart a run at t = 0). */
int mhd_set_time(mhd_handle h, double t);

/* Synchronise and return the current time and the last time step. */
int mhd_get_time(mhd_handle h, double* t, double* dt);

void mhd_destroy(mhd_handle h);

/* Message of the last error of this handle (or of the last failed
 * mhd_create when h is NULL).  Never NULL. */
const char* mhd_last_error(mhd_handle h);

/* ---- snapshots in the layout of the paper's HDF5 files (Sect. 5.3) ----
 *
 * var.h5: a scalar FP64 dataset `time`; group `data` with one dataset per
 * variable -- ax, ay, az, ux, uy, uz, lnrho, lnTT -- each of shape
 * [nz+6][ny+6][nx+6] (x fastest, i.e. the Fortran order (x, y, z) in which
 * the paper's files are read, the outer ghost layers kept), in the handle's
 * precision; group `grid` (x, y, z positions of the padded box, dx, dy, dz
 * with dz the mean vertical spacing, dx_1, dy_1, dz_1 the inverse spacing
 * per point -- on a non-uniform z grid the inverse of dz/dk -- and Lx, Ly,
 * Lz); group `settings` (`precision` = "S" or "D", nghost, nx, ny, nz, mx,
 * my, mz).  grid.h5: the groups `grid` and `settings` alone.  ln rho, ln T
 * and A are the full values (backgrounds added); x_i = (i - 3) dx, y alike,
 * z the layer positions.  The files are written in the HDF5 format without
 * the HDF5 library (superblock version 2, compact groups, contiguous
 * datasets; readable by HDF5 1.8 and later).
 *
 * mhd_write_snapshot: fills the ghosts of the current state (as a step's
 * first substep does), stages the padded state in the handle's RK
 * accumulator buffer (unused between steps) and writes var_path and/or
 * grid_path (either may be NULL, not both).  Synchronises the stream; one
 * field at a time passes through host memory.  Errors: MHD_ERR_ARG,
 * MHD_ERR_NONFINITE / MHD_ERR_TIMEOUT for a halted handle, MHD_ERR_CUDA,
 * MHD_ERR_IO (file not writable; a partial file may remain).
 *
 * mhd_h5_write: the same files from host data without a handle: p as for
 * mhd_create, t the time, padded the host state [8][nz+6][ny+6][nx+6] in
 * p->precision (may be NULL when var_path is NULL).  No CUDA call.
 *
 * mhd_h5_checksum: the checksum these files carry (Jenkins' lookup3
 * hashlittle with initial value 0) of len bytes at data; host only. */
int mhd_write_snapshot(mhd_handle h, const char* var_path, const char* grid_path);
int mhd_h5_write(const char* var_path, const char* grid_path, const mhd_params* p, double t, const void* padded);
unsigned int mhd_h5_checksum(const void* data, size_t len);

/* ---- diagnostics and kernel-level entry points (used by the tests) ---- */

/* Fill every ghost cell of the current state (rims, bottom/top rules and the
 * potential-field ghosts), as the first substep does. */
int mhd_fill_ghosts(mhd_handle h);

/* Copy the padded state (which = 0) or the RK accumulator (which = 1) as
 * [8][nz+6][ny+6][nx+6] (x fastest, ghosts included) into dst. */
int mhd_read_padded(mhd_handle h, int which, void* dst, int mem);

/* Evaluate the right-hand side of the current (ghost-filled) state at time t
 * and copy it as [8][nz+6][ny+6][nx+6] into dst (cells that carry no state
 * are zero).  Uses the accumulator buffer as scratch. */
int mhd_eval_rhs(mhd_handle h, double t, void* dst, int mem);

/* CFL time step of the current ghost-filled state (synchronising). */
int mhd_compute_dt(mhd_handle h, double* dt);

/* Diagnostics of the current ghost-filled state (synchronising). */
int mhd_compute_stats(mhd_handle h, mhd_stats* out);

/* Copy the vector potential of the driver magnetogram, A_x then A_y, as
 * [2][ny][nx] into dst. */
int mhd_read_target(mhd_handle h, void* dst, int mem);

/* ---- adjoint (gradients of a loss on the final state) ----
 *
 * The transposed linearisation of mhd_step with a frozen time step
 * (dt_fixed > 0; the CFL rule is not differentiable), for handles created
 * with params.adjoint = 1 and bc_z = 0.  Parameters: the driver magnetogram
 * B_z (through the inversion of Eq. 7 and the magnetic nudging of Sect. 2.1)
 * and the two driver velocity snapshots v0, v1 (through the velocity nudging
 * of Eq. 5 at the photosphere and in its three ghost layers).  Usage: save
 * checkpoints while stepping forward; seed the adjoint with dL/d(final
 * state); for each step in reverse order restore the state at its start and
 * call mhd_adjoint_step; read the gradients.  Reverse accumulation over many
 * steps with few checkpoints (binomial checkpointing) is scheduled by the
 * caller. */

/* Bytes of one checkpoint (the padded state, including the stateful
 * velocity ghosts). */
size_t mhd_checkpoint_bytes(mhd_handle h);

/* Copy the current state into dst (device memory of mhd_checkpoint_bytes)
 * and return its time in *t (synchronising). */
int mhd_save(mhd_handle h, void* dst, double* t);

/* Make a saved state (device memory) the current state at time t. */
int mhd_restore(mhd_handle h, const void* src, double t);

/* Start a reverse sweep: the state adjoint is set to lam ([8][nz][ny][nx],
 * dL/d(final state); zero in the ghost layers), the RK accumulator adjoint
 * and the parameter gradients to zero. */
int mhd_adjoint_init(mhd_handle h, const void* lam, int mem);

/* One reverse step: the current state (restored) is the state f_n at the
 * start of a step; the forward substeps are recomputed from it, then the
 * state adjoint is taken from step n+1 back to step n and the parameter
 * gradients are accumulated.  The forward state after the call is that of
 * f_n again (time undefined until the next mhd_restore). */
int mhd_adjoint_step(mhd_handle h);

/* Tapes: when device memory allows, a step's three substep input states are
 * kept instead of recomputed, so its reverse step reads them back (the
 * recomputation of forward substeps is then needed only when the state
 * history does not fit).  mhd_tape_bytes: bytes of one step's tape, three
 * state sets (3 x mhd_checkpoint_bytes) and 256 bytes for the step's start
 * time.
 * mhd_step_taped: one full RK step from the current state, exactly as
 * mhd_step(h, 1) computes it, that also leaves in `tape` (caller-owned
 * device memory of mhd_tape_bytes bytes, 256-byte aligned) the ghost-filled
 * state each of its three substeps read and the start time.  Asynchronous.
 * mhd_adjoint_step_taped: the reverse step of the step recorded in `tape`,
 * as mhd_adjoint_step computes it after restoring that step's first state,
 * without the forward recomputation; the handle's own state is not touched.
 * Asynchronous.  Both need the default FP32 kernels or MHD_RK_VARIANT=simple
 * (MHD_ERR_UNSUPPORTED otherwise); the adjoint one needs params.adjoint and
 * dt_fixed > 0 like mhd_adjoint_step. */
size_t mhd_tape_bytes(mhd_handle h);
int mhd_step_taped(mhd_handle h, void* tape);
int mhd_adjoint_step_taped(mhd_handle h, const void* tape);

/* Read the results of a reverse sweep: lam ([8][nz][ny][nx]) the adjoint of
 * the state at the sweep's current step (the velocity ghost adjoints folded
 * onto the photospheric layer, matching how mhd_create initialises them),
 * grad_bz ([ny][nx]), grad_v0, grad_v1 ([2][ny][nx]); any may be NULL. */
int mhd_adjoint_read(mhd_handle h, void* lam, void* grad_bz, void* grad_v0, void* grad_v1, int mem);

/* Loss helper: B_z = D1x A_y - D1y A_x on layer k of a state
 * ([8][nz][ny][nx], device) into out ([ny][nx], device), and the transpose:
 * given bbar ([ny][nx], device) write lam ([8][nz][ny][nx], device): zero
 * except A_x and A_y on layer k. */
int mhd_bz_plane(mhd_handle h, const void* state, int k, void* out);
int mhd_bz_plane_adjoint(mhd_handle h, const void* bbar, int k, void* lam);

/* ---- allocation-free variant ---- */

/* Vector potential A_x, A_y (Weyl gauge, A_z = 0) of the magnetogram bz, the
 * same result mhd_set_driver stores for its nudging target, for callers that
 * cannot allocate device memory and have no workspace to give: a host
 * application that reserves the whole GPU up front, a plugin inside a process
 * whose caching allocator already holds nearly all of HBM, or code that must
 * not pay for an allocation.  There is no counterpart in the paper; it is a
 * library convenience.
 *   nx, ny: powers of two in [8, 512]; larger sizes return MHD_ERR_ARG with a
 *     message (the scratch is a fixed 8 MiB + 24 KiB __device__ array that
 *     every GPU loading the library keeps until the process exits).
 *   dx, dy: grid spacings; precision: 32 or 64 (element type of bz, ax, ay).
 *   bz [ny][nx] input, ax, ay [ny][nx] outputs: device pointers owned by the
 *     caller.  stream: cudaStream_t (NULL: legacy default stream).
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Under CUDA's default lazy module loading that
 * first call is also what loads the library's module holding the array, so
 * the 8 MiB + 24 KiB are taken from the device then: a caller that reserves
 * all of the GPU's memory should make one call first (any size) and reserve
 * afterwards; later calls take nothing more.  The address is looked up again
 * if the device's context was destroyed and recreated (cudaDeviceReset).
 * All calls on a device share the one scratch array: calls that overlap on
 * the GPU (different streams, or different host threads) race and give wrong
 * results.  Asynchronous; errors are reported through mhd_last_error(NULL). */
int mhd_invert_magnetogram_static(int nx, int ny, double dx, double dy,
                                  int precision, const void* bz, void* ax,
                                  void* ay, void* stream);

/* ---- granulation driver (Sect. 2.3, Eqs. 1-4) ---- */

/* A generator of photospheric driver velocities that resemble granulation,
 * on a periodic nx x ny plane of spacings dx, dy, independent of any
 * simulation handle (the paper runs it as a 2D pre-step whose snapshots the
 * 3D model interpolates in time: pass two of its outputs to mhd_set_driver
 * as v0, v1).  All arithmetic is FP64 on the GPU.
 *
 * Granules sit on pixel centres, at most one per pixel.  Each carries its
 * birth time t0, lifetime T = lifetime (1 + lifetime_spread c_T), peak
 * amplitude v_max = v0 (1 + amp_spread c_v) (c_T, c_v: the caller's standard
 * normal draws at that pixel, clipped to [-1, 1]) and peak time
 * t_max = T sqrt(|ln(v_min / v_max)|) (Eq. 1), v_min = vmin_frac v0; its
 * amplitude is v(t) = v_max exp(-((t - t0 - t_max) / T)^2) (Eq. 2), equal to
 * v_min at birth and again at t0 + 2 t_max, when the granule dies.
 *
 * Lengths are in the units of dx, dy; times and speeds in any consistent
 * units (the paper's values: r_inner 0.64 Mm, r_granule 0.8 Mm, r_lane
 * 1.04 Mm, v0 1.028 km/s, vmin_frac 0.78, lifetime 5 min, spreads 0.10 and
 * 0.15, f_rot 5). */
typedef struct mhd_gran_params {
  double r_inner;          /* no new centre closer than this to a live one    */
  double r_granule;        /* the radial speed rises linearly to here ...      */
  double r_lane;           /* ... and falls as cos^2 to zero here (> r_granule) */
  double v0;               /* typical amplitude                                */
  double vmin_frac;        /* v_min / v0, in (0, 1 - amp_spread)               */
  double lifetime;         /* T_gran                                           */
  double lifetime_spread;  /* in [0, 1)                                        */
  double amp_spread;       /* in [0, 1)                                        */
  double f_rot;            /* amplification of the rotational part (Eq. 3)    */
} mhd_gran_params;

typedef struct mhd_gran_ctx* mhd_gran_handle;

/* Bytes of device workspace a generator needs (0 if the arguments are
 * invalid: nx, ny powers of two in [8, 1024]; dx, dy > 0; 0 < r_inner;
 * 0 < r_granule < r_lane; r_inner and r_lane below half the plane in each
 * direction and at most 64 pixels; the other parameters as stated above). */
size_t mhd_gran_workspace_bytes(int nx, int ny, double dx, double dy,
                                const mhd_gran_params* gp);

/* Create a generator with no granules.  workspace: caller-owned device
 * memory of mhd_gran_workspace_bytes() bytes, 256-byte aligned, kept alive
 * until mhd_gran_destroy.  stream: cudaStream_t (NULL: legacy default
 * stream) on which every launch of the generator is ordered.  Synchronises
 * the stream before returning.  Errors: mhd_last_error(NULL). */
int mhd_gran_create(int nx, int ny, double dx, double dy,
                    const mhd_gran_params* gp, void* workspace,
                    size_t ws_bytes, void* stream, mhd_gran_handle* out);

/* Advance the granule population to time t: remove every granule with
 * t - t0 - t_max > t_max (its amplitude has fallen below v_min after the
 * peak), then fill the plane: visiting the pixels by ascending
 * (keys[p], p), a granule starts at pixel p (t0 = t) when no live centre lies
 * closer than r_inner (nearest periodic image).  The result equals that
 * sequential visit exactly; the GPU reaches it in parallel rounds (a pixel
 * joins once no undecided pixel within r_inner precedes it), and the call
 * synchronises the stream once per round.
 *   keys [ny][nx] uint32, c_life, c_amp [ny][nx] double: the random draws
 *   (uniform keys, standard normals); mem: MHD_MEM_DEVICE or MHD_MEM_HOST.
 *   rounds (may be NULL): the parallel rounds taken.
 * The arrays are the caller's and may be reused when the call returns (host
 * arrays are staged into the workspace first).  Times passed to successive
 * calls should not decrease.  Errors: MHD_ERR_ARG (NULL generator or array,
 * bad mem flag, non-finite t), MHD_ERR_CUDA, MHD_ERR_TIMEOUT if the rounds
 * did not settle within nx ny + 1 (they cannot, by the argument above; the
 * population is then partly updated). */
int mhd_gran_update(mhd_gran_handle g, double t, const unsigned int* keys,
                    const double* c_life, const double* c_amp, int mem,
                    int* rounds);

/* The driver velocity v*_gran at time t (Eqs. 2-4) into v [2][ny][nx]
 * (vx, vy; float for precision 32, double for 64): the live granules'
 * radial fields, amplitude (Eq. 2) times the radial profile times the unit
 * vector from the centre, added where they overlap (v_gran); its
 * divergence-free part, times exp(-(2 |k| / k_N)^4) with
 * |k| / k_N = sqrt((k_x dx / pi)^2 + (k_y dy / pi)^2) and the mean and
 * Nyquist modes dropped (Eq. 3), times f_rot added back (v_vor); the sum
 * scaled by sqrt(<|v_gran|^2> / <|v_vor|^2>) (Eq. 4; zero if v_vor is).
 * v is the caller's (device or host per mem).  Asynchronous for device
 * output; host output returns once copied.  Errors: MHD_ERR_ARG (NULL
 * generator or v, precision not 32 or 64, bad mem flag, non-finite t),
 * MHD_ERR_CUDA. */
int mhd_gran_velocity(mhd_gran_handle g, double t, int precision, void* v,
                      int mem);

/* The granule maps: occ [ny][nx] int (1 where a granule is centred) and, if
 * par is not NULL, par [4][ny][nx] double (t0, T, v_max, t_max; zero where
 * occ is 0). */
int mhd_gran_read_granules(mhd_gran_handle g, int* occ, double* par, int mem);

/* Intermediate fields of the last mhd_gran_velocity, [2][ny][nx] double:
 * which = 0 the granular field v_gran, 1 the filtered rotational part
 * v_rot' of Eq. 3. */
int mhd_gran_read_field(mhd_gran_handle g, int which, double* dst, int mem);

/* Number of kernels this generator has launched since mhd_gran_create. */
long long mhd_gran_launch_count(mhd_gran_handle g);

/* The message of the generator's last error (NULL: of the last create). */
const char* mhd_gran_last_error(mhd_gran_handle g);

/* Frees host-side bookkeeping only (the workspace is the caller's). */
void mhd_gran_destroy(mhd_gran_handle g);

/* ---- instrumentation ---- */

/* Kernel classes timed by the profiler. */
#define MHD_KC_GHOST 0   /* pointwise ghost rules (and periodic copies)   */
#define MHD_KC_PFE 1     /* potential-field FFT, three kernels             */
#define MHD_KC_CFL 2     /* time-step reduction: partial maxima, finalize  */
#define MHD_KC_STATS 3   /* diagnostics: curl A, partial sums, finalize    */
#define MHD_KC_RK 4      /* fused right-hand side + RK update              */
#define MHD_NKC 5

/* enable != 0: from now on bracket every kernel class launched by mhd_step
 * with CUDA events on the stream it runs on; enable = 0 stops recording.
 * enable = 1: the step runs as usual, and classes that overlap (the first
 * substep's FFT on the side stream, the ghost rules and CFL reduction beside
 * it, the three FFT plane chains) are each timed in full, so the class times
 * of a step can sum to more than the step.  enable = 2: while recording,
 * every kernel runs on the handle's stream one after another (no side
 * streams), so the class times add up to the (slightly longer) step. */
int mhd_profile(mhd_handle h, int enable);

/* Synchronise, then return per class the summed event time in ms and the
 * number of kernel launches recorded since profiling was enabled, and reset
 * the record.  ms and launches point to MHD_NKC entries each. */
int mhd_read_profile(mhd_handle h, double* ms, long long* launches);

/* Number of kernels this handle has launched since mhd_create. */
long long mhd_launch_count(mhd_handle h);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
