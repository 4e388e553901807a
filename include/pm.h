/*
 * pm.h -- C ABI of the GB300 particle-mesh weak-lensing library.
 *
 * The library runs the forward model of MADLens (Boehm, Feng, Lee & Dai,
 * arXiv:2012.07266) on one GPU: FastPM-style kick-drift-kick particle-mesh
 * steps (Sec. 3), the Born lightcone projection with box replication,
 * rotation and the sub-evolution scheme onto convergence maps (Eq. conv,
 * Sec. 3), the PGD sharpening step (Sec. 3), and the reverse-mode derivative
 * of the maps with respect to the initial white-noise modes, Omega_m and
 * sigma_8 (Sec. 3, Appendix A).
 *
 * Conventions shared by every entry point:
 *  - Ownership: the caller allocates every device buffer, including the
 *    single workspace handed to pm_init; the library never allocates device
 *    memory.  Host-side bookkeeping (a few KB of tables) lives in the
 *    context and is freed by pm_destroy.
 *  - Streams: every call enqueues its kernels on the stream given to
 *    pm_init and returns without synchronising, except where stated
 *    (kappa_maps, pm_vjp and pm_sync_status synchronise that stream).
 *  - Errors: arguments are validated on the host before anything is
 *    enqueued; a failing check returns PM_ERR_ARG / PM_ERR_STATE /
 *    PM_ERR_WORKSPACE / PM_ERR_UNSUPPORTED and enqueues nothing.  A CUDA
 *    launch error returns PM_ERR_CUDA.  Non-finite values met on the device
 *    set a flag that the synchronising calls report as PM_ERR_NONFINITE; a
 *    bounded device-side wait for a bulk copy that gave up sets another
 *    flag, reported as PM_ERR_TIMEOUT.
 *  - Layouts: particle arrays are row-major (N, 3) with N = nc^3 and particle
 *    j = (jz * nc + jy) * nc + jx; meshes are [z][y][x] with x fastest;
 *    maps are [source][iy][ix] with ix along theta_x.
 *  - Units: H0 = 1, lengths in Mpc/h, momentum p = a^3 E(a) dx/da in Mpc/h.
 */
#ifndef PMLENS_PM_H
#define PMLENS_PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_ctx pm_ctx; /* opaque; created by pm_init, freed by pm_destroy */

typedef enum {
  PM_OK = 0,
  PM_ERR_ARG = 1,         /* invalid argument or configuration            */
  PM_ERR_WORKSPACE = 2,   /* workspace too small or misaligned            */
  PM_ERR_CUDA = 3,        /* a CUDA call or launch failed                 */
  PM_ERR_NONFINITE = 4,   /* NaN/Inf met on the device                    */
  PM_ERR_STATE = 5,       /* entry point called out of order              */
  PM_ERR_UNSUPPORTED = 6, /* size not supported by the FFT plans          */
  PM_ERR_TIMEOUT = 7      /* a device-side wait for an asynchronous copy
                             ran out of its iteration bound (the kernel
                             returned early; results are invalid)         */
} pm_status;

enum { PM_FP32 = 0, PM_FP64 = 1 };
enum { PM_MAX_ZS = 16 };

/*
 * Simulation parameters; mirrors the user parameters of the paper's Table 1
 * (BoxSize, Nmesh, B, Nsteps, N_maps, Nmesh2D, BoxSize2D, zs_source,
 * Omega_m, sigma_8, PGD, interpolation) plus the Eisenstein-Hu inputs of
 * Appendix A and the precision / checkpoint fields of this library.
 */
typedef struct {
  int32_t nc;              /* particles per side; N = nc^3                         */
  int32_t nmesh;           /* force mesh per side (B = nmesh / nc), <= 1024          */
  double box;              /* box side L, Mpc/h                                      */
  double omega_m, sigma8;  /* Table 1 cosmology                                      */
  double h, n_s, omega_b, t_cmb; /* Eisenstein-Hu transfer inputs (Appendix A)       */
  double a_init;           /* initial scale factor; steps are linear in a to 1       */
  int32_t nsteps;          /* number of kick-drift-kick steps                        */
  int32_t lpt_order;       /* 1 (Zel'dovich) or 2 (2LPT) initial conditions          */
  int32_t n_zs;            /* number of source planes, 1..PM_MAX_ZS                  */
  double zs[PM_MAX_ZS];    /* source redshifts (zs_source)                           */
  int32_t map_npix;        /* map pixels per side (Nmesh2D)                          */
  double map_fov_deg;      /* map side in degrees (BoxSize2D)                        */
  int32_t sub_evolution;   /* 1: sub-evolution projection ("interpolation")        */
  int32_t pgd;             /* 1: PGD sharpening of the projected positions           */
  double pgd_params[5];    /* alpha0, mu, k_l [h/Mpc], k_s [h/Mpc], n                */
  uint64_t rotation_seed;  /* seed of the per-replica rotation hash                  */
  int32_t rotate;          /* 1: rotate/shift each box replica                       */
  int32_t precision;       /* PM_FP32 (fast path) or PM_FP64 (plain comparator)      */
  int32_t ckpt_every;      /* adjoint checkpoint interval in steps; 0 = no adjoint;
                              >= nsteps: resident adjoint (every step kept, no
                              recompute in the reverse sweep)                        */
  int32_t jvp;             /* 1: keep the tangent state of pm_jvp                    */
} pm_config;

/* Device bytes the workspace of this configuration needs (its HBM footprint,
 * used for admission).  Returns PM_ERR_ARG / PM_ERR_UNSUPPORTED on a bad
 * configuration. */
pm_status pm_workspace_size(const pm_config* cfg, size_t* bytes);

/* Create a context.  Computes the FP64 cosmology tables on the host (linear
 * growth, FastPM time factors, comoving distance, Eisenstein-Hu P(k)) and
 * uploads them into the workspace.  d_workspace: device buffer of at least
 * pm_workspace_size() bytes, 256-byte aligned, owned by the caller and kept
 * alive until pm_destroy.  stream: a cudaStream_t (NULL = legacy stream). */
pm_status pm_init(pm_ctx** out, const pm_config* cfg, void* d_workspace, size_t bytes,
                  void* stream);

/* Initial conditions (Sec. 3/Appendix A: Gaussian modes, EH power, LPT):
 * d_noise is the caller's real-space N(0,1) white-noise field on the nc^3
 * lattice, [z][y][x] float64 on the device.  delta_L(k) = DFT(noise) *
 * sqrt(P(k) nc^3 / L^3); Zel'dovich (and 2LPT) displacements place the
 * particles at a_init; the PM force at those positions is computed so that
 * pm_step(0) can kick.  Resets the maps. */
pm_status pm_ic(pm_ctx* ctx, const double* d_noise);

/* One FastPM step i (0 <= i < nsteps, in order; Sec. 3): kick p to
 * a_{i+1/2} with the force at a_i, drift x to a_{i+1}, paint, FFT Poisson and
 * gradient, inverse FFT to the force at a_{i+1}; with PGD on and shell i
 * inside the lightcone, also the PGD displacement meshes. */
pm_status pm_step(pm_ctx* ctx, int32_t i);

/* Project shell i (chi(a_{i+1}), chi(a_i)] onto the internal FP64 maps
 * (Eq. conv with Born weights, box replication and rotation, sub-evolution
 * and PGD as configured).  Must follow pm_step(i) directly; a shell beyond
 * the farthest source is a no-op. */
pm_status lens_project(pm_ctx* ctx, int32_t i);

/* Write the convergence maps kappa = sum of projected weights minus the
 * mean-density term (Eq. conv) to d_maps: n_zs * npix^2 float64, device,
 * caller-owned.  Synchronises the stream; PM_ERR_NONFINITE if any map value
 * or projected position was not finite. */
pm_status kappa_maps(pm_ctx* ctx, double* d_maps);

/* Reverse-mode derivative of a scalar loss of the maps (Sec. 3, VJP;
 * Appendix A for Omega_m, sigma_8).  Requires ckpt_every > 0 and the whole
 * forward run (pm_ic, all pm_step / lens_project) done.  d_dL_dkappa:
 * n_zs * npix^2 float64 (device); d_dL_dnoise: nc^3 float64 output
 * (device); h_dL_dparams: 2 float64 on the HOST, [dL/dOmega_m, dL/dsigma_8]
 * (either output pointer may be NULL).  Synchronises the stream. */
pm_status pm_vjp(pm_ctx* ctx, const double* d_dL_dkappa, double* d_dL_dnoise,
                 double* h_dL_dparams);

/* Replace source plane s (0 <= s < n_zs) by a distribution of source
 * redshifts (Eq. conv with a general n(chi')): n tabulated at npts >= 2
 * strictly ascending redshifts h_z (host arrays, 0 < z < 1/a_init - 1),
 * n >= 0, linear in between and zero outside, normalised to unit integral.
 * Map s then weights each projected particle by the lensing efficiency
 * q(chi) = int dz' n(z') (1 - chi / chi(z'))_+ instead of (chi_s - chi)/chi_s,
 * and its mean-density term becomes (3/2) Om (H0/c)^2 int chi q / a dchi.
 * Builds the host FP64 tables (and their Omega_m +/- h versions when the
 * derivatives are configured).  Call after pm_init and before the first
 * lens_project of a run (PM_ERR_STATE otherwise); PM_ERR_ARG on invalid
 * tables.  Synchronises the stream. */
pm_status pm_set_source_nz(pm_ctx* ctx, int32_t s, const double* h_z, const double* h_n, int32_t npts);

/* Forward-mode derivative (JVP) of the maps along a direction of the initial
 * white noise (Sec. 3: the model is differentiable in the initial modes; the
 * paper checks its Jacobian-vector product by changing the initial field in
 * one pixel, Fig. 8).  Runs the whole forward model from d_noise (pm_ic, every
 * pm_step and lens_project) with the tangent state carried alongside, and
 * writes the maps (as kappa_maps) to d_kappa and their derivative along
 * d_dnoise to d_dkappa.  d_noise, d_dnoise: nc^3 float64 (device, [z][y][x]);
 * d_kappa, d_dkappa: n_zs * npix^2 float64 outputs (device, caller-owned).
 * Requires cfg->jvp = 1 (PM_ERR_UNSUPPORTED otherwise).  The context is left
 * as after a full forward run (a pm_vjp may follow when ckpt_every > 0).
 * Synchronises the stream; PM_ERR_NONFINITE as kappa_maps. */
pm_status pm_jvp(pm_ctx* ctx, const double* d_noise, const double* d_dnoise, double* d_kappa, double* d_dkappa);

/* Shot-noise run (Sec. 4, Fig. accuracy: the shot noise of the maps is
 * estimated from runs with randomly placed particles, whose averaged power
 * spectrum is subtracted).  Places the nc^3 particles i.i.d. uniform in the
 * box -- coordinate k of particle j from output 3j + k of the SplitMix64
 * sequence seeded with `seed` (output n mixes the state
 * seed + (n + 1) * 0x9E3779B97F4A7C15), its top 24 bits r giving x = L r / 2^24
 * -- with zero momentum and without PGD, projects every shell of the
 * lightcone as lens_project would (replicas, rotations, source planes or
 * distributions), subtracts the mean-density terms and writes the maps
 * (n_zs * npix^2 float64, device, caller-owned, layout as kappa_maps) to
 * d_kappa.  The context's particle state, maps and derivative records are
 * overwritten: pm_step, lens_project, kappa_maps, pm_vjp and the inspection
 * calls return PM_ERR_STATE until the next pm_ic.  Synchronises the stream;
 * PM_ERR_NONFINITE as kappa_maps. */
pm_status pm_shot_noise_maps(pm_ctx* ctx, uint64_t seed, double* d_kappa);

/* Workspace bytes pm_map_cl needs for nmaps maps of npix^2 pixels and nbins
 * bins (PM_ERR_ARG where pm_map_cl would refuse the sizes). */
pm_status pm_map_cl_workspace_size(int32_t npix, int32_t nmaps, int32_t nbins, size_t* bytes);

/* Binned flat-sky angular power spectrum of maps (Sec. 4, Fig. accuracy: the
 * convergence power spectra and the shot noise subtracted from them).  Needs
 * no context.  For map m (d_maps + m npix^2, float64 [iy][ix], device) and
 * every DFT mode (m_x, m_y), each in -npix/2 .. npix/2 - 1, with
 * FOV_rad = fov_deg * (pi / 180) and Omega_pix = (FOV_rad / npix)^2:
 *   C = Omega_pix |sum_j kappa_j exp(-2 pi i (m_x ix + m_y iy) / npix)|^2 / npix^2,
 *   l = (2 pi / FOV_rad) * sqrt(m_x^2 + m_y^2)   (IEEE double, in this order);
 * the value of bin b is the mean of C over the modes with
 * h_edges[b] <= l < h_edges[b+1] (0 for a bin without modes), and
 *   d_cl[m * nbins + b] = beta * d_cl[m * nbins + b] + alpha * value
 * (beta = 0 ignores the old contents; beta = 1, alpha = -1/R subtracts the mean
 * of R spectra, e.g. of shot-noise runs).  npix a power of two in [8, 4096],
 * 1 <= nmaps, 1 <= nbins <= 2048, h_edges (host, nbins + 1 values) strictly
 * ascending (the last may be +inf), fov_deg > 0: PM_ERR_ARG otherwise.
 * d_workspace: device, 256-byte aligned, at least pm_map_cl_workspace_size
 * bytes (PM_ERR_WORKSPACE otherwise).  h_counts: NULL, or host int64[nbins]
 * receiving the number of modes of each bin (the call then synchronises the
 * stream).  Enqueued on `stream` (a cudaStream_t; NULL: the legacy default
 * stream).  FP64 throughout. */
pm_status pm_map_cl(const double* d_maps, int32_t nmaps, int32_t npix, double fov_deg, const double* h_edges,
                    int32_t nbins, double alpha, double beta, double* d_cl, int64_t* h_counts, void* d_workspace,
                    size_t workspace_bytes, void* stream);

/* Free the context (not the caller's workspace). */
pm_status pm_destroy(pm_ctx* ctx);

/* Static description of a status code. */
const char* pm_strerror(pm_status status);

/* ---- inspection entry points (state transfer for tests and users) ----- */

/* Current particles: positions in [0, L) and momenta, (N, 3) float64 on the
 * device (either pointer may be NULL).  After pm_step(i): x(a_{i+1}),
 * p(a_{i+1/2}). */
pm_status pm_get_particles(pm_ctx* ctx, double* d_x, double* d_p);

/* Replace the particle state by (N, 3) float64 device arrays, taken as the
 * state after step `next_step - 1` (x at a_{next_step}, p at a_{next_step-1/2};
 * next_step = 0 means the initial state at a_init), and compute the force at
 * those positions. */
pm_status pm_set_particles(pm_ctx* ctx, const double* d_x, const double* d_p,
                           int32_t next_step);

/* PM force F = -(3/2) Omega_m grad(phi) (Mpc/h, momentum units per unit
 * kick factor) at the current particle positions, (N, 3) float64 device. */
pm_status pm_get_forces(pm_ctx* ctx, double* d_f);

/* PGD displacement (Mpc/h) at the current positions, (N, 3) float64 device;
 * valid after pm_step(i) of a shell inside the lightcone with PGD on. */
pm_status pm_get_pgd(pm_ctx* ctx, double* d_s);

/* Forward r2c DFT (sign -1, unnormalised) of a real nmesh^3 float64 field
 * [z][y][x] into d_out: nmesh * nmesh * (nmesh/2 + 1) complex as interleaved
 * float64 [z][y][kx][re,im], through the library's FFT kernels. */
pm_status pm_fft_r2c(pm_ctx* ctx, const double* d_in, double* d_out);

/* CIC density (mean 1) of the current particles on the force mesh,
 * nmesh^3 float64 device [z][y][x]. */
pm_status pm_get_density(pm_ctx* ctx, double* d_rho);

/* Synchronise the stream and report the sticky device error flag. */
pm_status pm_sync_status(pm_ctx* ctx);

/* ---- instrumentation (no counterpart in the paper) --------------------- */

/* Turn per-kernel CUDA-event timing on (1) or off (0).  Kernel launches are
 * always counted per kernel class; with timing on, each launch is bracketed
 * by two events recorded on the context's stream.  Synchronises the stream. */
pm_status pm_profile(pm_ctx* ctx, int32_t enable);

/* Per-class totals since the last read, each a host array of nkinds
 * entries (any pointer may be NULL): kernel time in ms (0 unless timing was
 * on), launch counts, and algorithmic HBM bytes of those launches (the bytes
 * the operation must move: each pass's input read and output written once,
 * gathered meshes once, particle state once).  Synchronises the stream, then
 * resets the counters. */
pm_status pm_profile_read(pm_ctx* ctx, double* ms, int64_t* launches, double* bytes, int32_t nkinds);

/* Number of kernel classes and the static name of class `kind`. */
int32_t pm_kernel_kinds(void);
const char* pm_kernel_name(int32_t kind);

/* ---- allocation-free variant (no counterpart in the paper) -------------- */

/* PM forces F = -(3/2) Omega_m grad(phi) at n particles, like pm_set_particles
 * followed by pm_get_forces, but without a context or a workspace: for callers
 * that cannot allocate device memory (code inside a framework whose allocator
 * owns the device memory, plugins or callbacks that must not allocate,
 * processes under a hard device-memory budget).  Its scratch meshes live in a
 * file-scope device array of about 10 MB that every GPU loading the library
 * holds until the process exits.
 *  d_x: (n, 3) float64 positions in [0, box) Mpc/h, device, caller-owned.
 *  d_f: (n, 3) float64 forces out (Mpc/h per unit kick factor), device.
 *  nmesh: force mesh per side, one of 32 or 64 (larger meshes return
 *         PM_ERR_UNSUPPORTED before any device work); each particle carries
 *         mass nmesh^3 / n so that the mean density is 1.  FP32 arithmetic.
 *  stream: cudaStream_t on which the work is enqueued; the call does not
 *          synchronise.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and caches it.  With CUDA's lazy module
 * loading the library's device code, and with it this array, is created on a
 * device at the first call or kernel launch of the library there, so that
 * first call may itself take device memory: make it before a hard memory
 * budget is reached and before any stream capture.  The cached address does
 * not survive cudaDeviceReset: do not call this entry point on a device that
 * was reset after its first call.  No cudaMalloc/cudaFree or allocating
 * library routine is called.
 * Every call shares the one array (its previous contents are overwritten;
 * the density is cleared on each call), so calls that overlap on the GPU --
 * on different streams or from different threads -- race and must be
 * serialised by the caller. */
pm_status pm_forces_static(const double* d_x, int64_t n, int32_t nmesh, double box, double omega_m,
                           double* d_f, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PMLENS_PM_H */
