// Internal declarations of the PM lensing library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/pm.h"

namespace pmlens {

constexpr double kCoverH0 = 2997.92458;  // c / H0 in Mpc/h
constexpr int kMaxReplicas = 96;         // replicas per lens launch (more -> several launches)
constexpr int kChiTab = 16384;           // entries of the chi -> (D1, 1/a) tables

// ---------------------------------------------------------------- cosmology
// FP64 background on the host: linear growth by RK4 in ln a with cubic
// Hermite interpolation, comoving distance, Eisenstein-Hu linear power.
struct Cosmo {
  double om, s8, h, ns, ob, tcmb;
  // tables on a uniform ln a grid
  double lna0, dlna;
  int n;
  std::vector<double> d1, d1d, d2, d2d, chi;  // D1, dD1/dlna, D2, dD2/dlna, chi
  double pk_norm;

  void init(double omega_m, double sigma8, double hh, double n_s, double omega_b, double t_cmb);
  double E(double a) const;
  double dlnE_dlna(double a) const;
  void state(double a, double* D1, double* dD1, double* D2, double* dD2) const;
  double D1(double a) const;
  double D2(double a) const;
  double gp(double a) const;   // a^3 E dD1/da
  double gp2(double a) const;  // a^3 E dD2/da
  double gf(double a) const;   // a^2 E dgp/da
  double chi_a(double a) const;
  double a_of_chi(double c) const;
  void a_of_chi_grid(double h, int n, double* out) const;  // a(q h), q < n, O(n) sweep
  double transfer(double k_hmpc) const;  // Eisenstein & Hu (1998) with BAO
  double pk(double k_hmpc) const;        // sigma8-normalised linear P(k), z = 0
};

// per-replica transform, packed for kernel parameters
struct Replica {
  int16_t n[3];      // replica offsets (units of the box)
  int16_t shift[3];  // periodic shift in force-mesh cells
  uint8_t perm[3];   // new axis d takes old axis perm[d]
  uint8_t flip;      // bit d: flip axis d
};

struct LensShell {
  double chi_lo2, chi_hi2; // squared shell bounds (Mpc/h)^2
  double d1_next, gp_half; // D1(a_{i+1}), g_p(a_{i+1/2})
  int nrep;
  Replica rep[kMaxReplicas];
};

// Path-precision (R) and FP32 copies of a projection's FP64 scalar parameters,
// rounded once on the host: on this GPU FP64 instructions, conversions
// included, run at a small fraction of the FP32 rate, so the kernels' hot loops
// take these copies instead of converting the FP64 fields at each use.
template <typename R>
struct GeomMirrors {
  R cell_len, lo2, hi2, fov_half, inv_dtheta, tan_half, margin, tab_hinv;
  float cull_cell_len, cull_lo2, cull_hi2, cull_tan_half, cull_margin;
};

template <typename R>
inline GeomMirrors<R> geom_mirrors(double cell_len, double lo2, double hi2, double fov_half, double inv_dtheta,
                                   double tan_half, double margin, double tab_hinv) {
  GeomMirrors<R> g;
  g.cell_len = (R)cell_len; g.lo2 = (R)lo2; g.hi2 = (R)hi2; g.fov_half = (R)fov_half;
  g.inv_dtheta = (R)inv_dtheta; g.tan_half = (R)tan_half; g.margin = (R)margin; g.tab_hinv = (R)tab_hinv;
  g.cull_cell_len = (float)cell_len; g.cull_lo2 = (float)lo2; g.cull_hi2 = (float)hi2;
  g.cull_tan_half = (float)tan_half; g.cull_margin = (float)margin;
  return g;
}

// kernel classes for launch counting and optional event timing
enum KernelKind {
  KK_KDK_PAINT = 0, KK_PAINT, KK_FFT_X_FWD, KK_FFT_Y_FWD, KK_FFT_Z_FWD, KK_FFT_Z_OP, KK_FFT_Y_INV,
  KK_FFT_X_INV, KK_LENS, KK_IC, KK_MISC, KK_ADJ, KK_ADJ_FFT, KK_ADJ_LENS, KK_JVP, KK_ADJ_PAINT, KK_ADJ_READ,
  KK_COUNT
};
const char* kernel_kind_name(int k);

// Per-context launch counter and CUDA-event timer.  When timing is on, each
// launch is bracketed by two events recorded on the launching stream; the
// elapsed times are resolved on read.
struct Prof {
  bool timing = false;
  long long launches[KK_COUNT] = {};
  double ms[KK_COUNT] = {};
  double bytes[KK_COUNT] = {};  // algorithmic HBM bytes of the counted launches
  long long timed[KK_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  cudaEvent_t get();
  void resolve();
  ~Prof();
};

struct ProfScope {
  Prof* p;
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(Prof* p_, int k, cudaStream_t s_, double algo_bytes = 0.0);
  ~ProfScope();
};

// chi-grid tables (FP64 in the workspace, FP32 mirrors for the FP32 path)
enum TabId { T_D1 = 0, T_INVA, T_DD1, T_DINVA, T_D1P, T_D1M, T_INVAP, T_INVAM, T_COUNT };

// workspace layout (byte offsets)
struct Layout {
  size_t cell, frac, mom, fmesh, smesh, maps, flags, sqrtp, tab_d1, tab_inva;
  size_t pid, cell2, frac2, mom2, pid2, sort_cnt;  // original index, sort double buffer, bucket counts
  size_t scratch;  // start of the scratch union
  // step scratch
  size_t rho, cbuf, ubuf;
  // IC scratch (aliases step scratch)
  size_t ic_real, ic_cbuf, ic_u, ic_out;
  // adjoint storage (ckpt_every > 0)
  size_t adj;
  size_t state_bytes;       // one particle state: cell | frac x3 | mom x3
  size_t tan_x, tan_p, tan_tmp, tan_f, tan_s, tan_maps, tan_ic;
  size_t qtab, qtab_f;  // lensing efficiency tables of n(z) sources: FP64 and FP32 mirror
  size_t adj_noise, adj_ckpt, adj_seg, adj_fseg, adj_sseg, adj_lx, adj_lp, adj_v, adj_vs, adj_paint, adj_ic;
  size_t adj_lam;  // FP32 path: dL/dkappa rounded to FP32 for the projection transposes
  size_t tab_dd1, tab_dinva, tab_d1p, tab_d1m, tab_invap, tab_invam, sqrtp_p, sqrtp_m, adj_acc;
  int nck, nic;             // checkpoints, IC adjoint fields
  size_t ftab;              // FP32 mirrors of the chi tables (TabId order)
  size_t total;
};

}  // namespace pmlens

struct pm_ctx {
  pm_config cfg;
  cudaStream_t stream;
  int prec;        // PM_FP32 / PM_FP64
  int rsz;         // sizeof(real)
  int nc, M;       // particle grid, mesh
  long long np;    // particles
  int P, Pc;       // complex row pitch (mesh, particle grid)
  long long mesh_elems, cmesh_elems, cgrid_elems;
  int nout_step;   // complex outputs of the step's spectral pass (3 or 6)
  char* ws;
  size_t ws_bytes;
  pmlens::Layout L;
  pmlens::Cosmo cosmo;
  std::vector<double> a, ah, kick, drift;
  std::vector<double> chi_a;   // chi(a_i)
  std::vector<double> chi_s;   // source distances
  double chi_tab_max, chi_tab_h;
  double mean_term[PM_MAX_ZS];
  // Omega_m +/- h copies of the cosmology-dependent coefficients (adjoint)
  double adj_h;
  pmlens::Cosmo cos_p, cos_m;
  std::vector<double> kick_p, kick_m, drift_p, drift_m, chi_s_p, chi_s_m;
  double mean_p[PM_MAX_ZS], mean_m[PM_MAX_ZS];
  // source distributions (pm_set_source_nz): bit s set when source s is n(z)
  unsigned nz_mask = 0;
  std::vector<double> nz_z[PM_MAX_ZS], nz_n[PM_MAX_ZS];
  int next_step;     // next pm_step index; -1 before pm_ic
  int last_stepped;  // index of the last pm_step, -1 none
  int projected;     // last projected shell
  int pgd_valid;     // PGD meshes valid for last_stepped
  size_t s_at = 0;   // workspace offset of the PGD meshes the lens kernels read (0: L.smesh)
  size_t f_at = 0;   // workspace offset of the current force meshes (0: L.fmesh)
  std::vector<char> sorted_after;  // resident adjoint: the state was re-sorted at the end of step i
  const double* tan_noise = nullptr;  // pm_jvp: noise direction for the tangent initial conditions
  int tan_on = 0;                     // pm_jvp: the tangent state follows the particle order
  int ic_done;
  int vjp_state_lost;  // 1: checkpoints do not describe the current run
  pmlens::Prof prof;
};

namespace pmlens {

// ---------------------------------------------------------------- launchers
// FFT (fft.cu)
inline bool fft_supported(int n) {
  switch (n) {
    case 32: case 64: case 96: case 128: case 192: case 256: case 512: case 1024: return true;
    default: return false;
  }
}
// real [n][n][n] -> spectrum [n][n][P] (forward, sign -1, unnormalised)
// err: timeout word of the TMA-pipelined column passes (null: plain passes
// without device-side waits)
template <typename R>
cudaError_t fft3d_r2c(const R* real, void* cplx, int n, int P, cudaStream_t s, Prof* prof, int* err);
// spectral operators applied in the fused z pass: out_o = mult_o(k) * spectrum
enum SpecOp { OP_FORCE = 0, OP_FORCE_PGD = 1, OP_LPT1 = 2, OP_LPT2_DERIV = 3, OP_GRAD_NEG = 4,
              OP_IDENTITY = 5 };
struct SpecParams {
  int op;
  double kf;        // 2 pi / L
  double scale;     // global factor (includes 1/n^3)
  double pgd_scale; // alpha * (M/L) / n^3
  double kl, ks, nexp;
  const double* sqrtp;  // table indexed by integer |n|^2 (OP_LPT*)
  int* err;             // timeout word of the TMA column passes (null: plain passes)
};
// forward x,y passes of `real`, fused z pass (forward, multiply, inverse) into
// nout complex buffers, then inverse y,x passes into the real outputs.
// kind >= 0 books every launch under that class (e.g. KK_IC), else per pass.
template <typename R>
cudaError_t spectral_apply(const R* real_in, void* cbuf, void* const* ubufs, R* const* real_out,
                           int nout, int n, int P, const SpecParams& sp, cudaStream_t s, Prof* prof,
                           int kind = -1);

// particles (particles.cu)
template <typename R>
cudaError_t launch_ic_particles(pm_ctx* c, R* const* psi1, R* const* psi2, double d1, double d2,
                                double gp1, double gp2);
template <typename R>
cudaError_t launch_paint(pm_ctx* c, R* rho);
template <typename R>
cudaError_t launch_kdk_paint(pm_ctx* c, R* rho, double ckick, double cdrift);
template <typename R>
cudaError_t launch_readout(pm_ctx* c, R* const* meshes, double scale, double* out);
template <typename R>
cudaError_t launch_set_particles(pm_ctx* c, const double* x, const double* p);
template <typename R>
cudaError_t launch_random_particles(pm_ctx* c, uint64_t seed);
template <typename R>
cudaError_t launch_get_particles(pm_ctx* c, double* x, double* p);
template <typename R>
cudaError_t launch_lpt2_source(pm_ctx* c, R* const* d, R* src, long long n);
template <typename R>
cudaError_t launch_convert_in(const double* in, R* out, long long n, cudaStream_t s, Prof* pf);
template <typename R>
cudaError_t launch_convert_out(const R* in, double* out, long long n, double scale, cudaStream_t s, Prof* pf);

// spatial sort (sort.cu)
void launch_iota(pm_ctx* c);
template <typename R>
cudaError_t sort_particles(pm_ctx* c);
template <typename R>
cudaError_t launch_unpermute3(pm_ctx* c, const R* src, const uint32_t* pid, R* dst);
template <typename R>
cudaError_t launch_permute3(pm_ctx* c, const R* src, const uint32_t* pid, R* dst);
size_t sort_scratch_bytes(int M);
// Resident adjoint (ckpt_every >= nsteps): the forward keeps every step's state, force meshes and
// PGD meshes in the workspace, and the reverse sweep recomputes nothing.
inline bool adj_resident(const pm_config& cfg) { return cfg.ckpt_every > 0 && cfg.ckpt_every >= cfg.nsteps; }
// re-sort every 4 steps; with checkpoint segments, only at segment boundaries
inline int sort_every(const pm_config& cfg) {
  return cfg.ckpt_every > 0 && cfg.ckpt_every < cfg.nsteps ? cfg.ckpt_every : 4;
}

// lensing (lens.cu)
template <typename R>
cudaError_t launch_lens(pm_ctx* c, const LensShell& sh, int use_pgd);
cudaError_t launch_kappa_finalize(pm_ctx* c, double* out);

// helpers
inline char* ws_ptr(pm_ctx* c, size_t off) { return c->ws + off; }

// chi table `id` in the path's precision R (FP64 workspace copy or FP32 mirror)
template <typename R>
inline const R* chi_table(pm_ctx* c, int id) {
  if constexpr (sizeof(R) == 8) {
    size_t off = 0;
    switch (id) {
      case T_D1: off = c->L.tab_d1; break;
      case T_INVA: off = c->L.tab_inva; break;
      case T_DD1: off = c->L.tab_dd1; break;
      case T_DINVA: off = c->L.tab_dinva; break;
      case T_D1P: off = c->L.tab_d1p; break;
      case T_D1M: off = c->L.tab_d1m; break;
      case T_INVAP: off = c->L.tab_invap; break;
      default: off = c->L.tab_invam;
    }
    return reinterpret_cast<const R*>(c->ws + off);
  } else {
    return reinterpret_cast<const R*>(c->ws + c->L.ftab + (size_t)id * ((kChiTab * 4 + 255) & ~size_t(255)));
  }
}
inline int* flags_ptr(pm_ctx* c) { return reinterpret_cast<int*>(c->ws + c->L.flags); }
inline int* timeout_ptr(pm_ctx* c) { return flags_ptr(c) + 1; }
// particles whose PGD displacement the projection gathered since the last profile read
// (they bound the mesh bytes its gathers must move)
inline unsigned long long* lens_gather_count(pm_ctx* c) {
  return reinterpret_cast<unsigned long long*>(c->ws + c->L.flags + 64);
}
// q tables of the n(z) sources, kind 0: q(chi), 1: dq/dchi, 2: q at Omega_m + h, 3: at
// Omega_m - h; n_zs * kChiTab entries per kind (source s at s * kChiTab)
enum QKind { Q_CENTRAL = 0, Q_DERIV = 1, Q_PLUS = 2, Q_MINUS = 3 };
template <typename R>
inline const R* qtable(pm_ctx* c, int kind) {
  const size_t n = (size_t)c->cfg.n_zs * kChiTab;
  if constexpr (sizeof(R) == 8) return reinterpret_cast<const R*>(c->ws + c->L.qtab) + kind * n;
  else return reinterpret_cast<const R*>(c->ws + c->L.qtab_f) + kind * n;
}
inline size_t fmesh_at(const pm_ctx* c) { return c->f_at ? c->f_at : c->L.fmesh; }
inline size_t smesh_at(const pm_ctx* c) { return c->s_at ? c->s_at : c->L.smesh; }

}  // namespace pmlens
