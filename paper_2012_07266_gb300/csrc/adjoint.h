// Internal declarations of the adjoint kernels (adjoint.cu) and of the
// transposed spectral pass (fft.cu).
#pragma once

#include "pm_internal.h"

namespace pmlens {

template <typename R>
struct AdjState {
  const uint32_t* cell;
  const R *fx, *fy, *fz, *px, *py, *pz;
};

template <typename R>
struct LensAdjArgs {
  AdjState<R> st;
  const R *S0, *S1, *S2;  // PGD displacement meshes (cells), or null
  long long np;
  int M;
  double cell_len, chi_lo2, chi_hi2, fov_half, inv_dtheta, tan_half, margin;
  int npix, nzs, sub;
  double chi_s[PM_MAX_ZS];
  double wpref, d1_next, inv_gp_half, tab_hinv;
  R chi_s_r[PM_MAX_ZS], wpref_r, d1_next_r, inv_gp_half_r;  // the same rounded to R on the host
  GeomMirrors<R> g;                                          // the geometry scalars rounded to R
  int tab_n;
  const R *tab_d1, *tab_dd1, *tab_inva, *tab_dinva;  // path precision
  unsigned nz_mask;         // bit s: source s is a distribution n(z)
  const R *qtab, *dqtab;    // its q(chi) and dq/dchi, n_zs x tab_n
  const R* lam;       // dL/dkappa, n_zs * npix^2, in the path precision
  R* lx;              // d/dx accumulators (cells), 3 * np
  R* lp;              // d/dp accumulators (cells), 3 * np
  R* vS;              // d/dS out (cells), 3 * np, or null
  int nrep;
  Replica rep[kMaxReplicas];
};

// sum over nin real inputs of conj(multiplier_{first + c}) * DFT(input_c), then
// inverse transform into `real_out` (the transpose of spectral_apply's
// outputs first .. first + nin - 1 for the same SpecParams).
template <typename R>
cudaError_t spectral_transpose(R* const* real_in, int nin, int first, void* const* ubufs, void* cbuf, R* real_out,
                               int n, int P, const SpecParams& sp, cudaStream_t s, Prof* prof);

// the same with inputs i < npre already x,y-transformed in ubufs[i] (by spectral_forward_xy)
template <typename R>
cudaError_t spectral_transpose_pre(R* const* real_in, int nin, int npre, int first, void* const* ubufs, void* cbuf,
                                   R* real_out, int n, int P, const SpecParams& sp, cudaStream_t s, Prof* prof);

// x and y forward passes of nin real inputs into the half spectra ubufs[i]
template <typename R>
cudaError_t spectral_forward_xy(R* const* real_in, int nin, void* const* ubufs, int n, int P, const SpecParams& sp,
                                cudaStream_t s, Prof* prof);

// the same for the first nl values of each cell of an FP32 mesh interleaved per cell
// with `lanes` values (lanes 4: nl 3 or 4; lanes 2: nl 2), into ubufs[0 .. nl-1] (FP32
// only; other combinations and the FP64 path return cudaErrorInvalidValue)
template <typename R>
cudaError_t spectral_forward_xy_il(const R* il, int lanes, int nl, void* const* ubufs, int n, int P,
                                   const SpecParams& sp, cudaStream_t s, Prof* prof);

// paint three cotangent components v (3 x np) into one FP32 mesh interleaved per cell as
// float4 (x, y, z, unused): one 16-byte vector reduction per corner
void adj_paint_weights4(const AdjState<float>& s, const float* v, float* mesh4, int M, long long np, cudaStream_t st,
                        Prof* pf);
// paint two cotangent sets at the same positions, v and w (3 x np each): v_x, v_y, v_z, w_x
// into the float4-interleaved mesh4, w_y, w_z into the float2-interleaved mesh2
void adj_paint_weights6(const AdjState<float>& s, const float* v, const float* w, float* mesh4, float* mesh2, int M,
                        long long np, cudaStream_t st, Prof* pf);

template <typename R>
void adj_paint_weights(const AdjState<R>& s, const R* v, R* const* meshes, int M, long long np, cudaStream_t st,
                       Prof* pf);
template <typename R>
void adj_readout_grad(const AdjState<R>& s, R* const* meshes, const R* v, const R* phi, double mass, R* lx,
                      const R* lp, double* dot, int M, long long np, cudaStream_t st, Prof* pf);
// two transposes at the same positions in one pass: lam_x += sum_c v_c grad readout(mesh_c)
// + sum_c w_c grad readout(mesh2_c) + mass grad readout(phi); dot = sum_j lp_j . readout(mesh)(x_j)
template <typename R>
void adj_readout_grad2(const AdjState<R>& s, R* const* meshes, const R* v, R* const* meshes2, const R* w,
                       const R* phi, double mass, R* lx, const R* lp, double* dot, int M, long long np, cudaStream_t st,
                       Prof* pf);
template <typename R>
void adj_axpy(R* y, const R* x, double a, long long n, cudaStream_t st, Prof* pf);
template <typename R>
void adj_scale(R* y, const R* x, double a, long long n, cudaStream_t st, Prof* pf);
template <typename R>
void adj_dot(const R* a, const R* b, long long n, double* acc, cudaStream_t st, Prof* pf);
void adj_dsum(const double* a, long long n, double* acc, cudaStream_t st, Prof* pf);
template <typename R>
void adj_combine2(const R* lx, const R* lp, R* const* outs, double ca, double cb, double scale, long long n,
                  cudaStream_t st, Prof* pf);
template <typename R>
void adj_ic_dot(const R* lx, const R* lp, R* const* psi1, R* const* psi2, double d1, double d2, double g1, double g2,
                double cpl, long long n, double* acc, cudaStream_t st, Prof* pf);
template <typename R>
void adj_lpt2_src(const R* ls, R* const* d, R* const* out, long long n, cudaStream_t st, Prof* pf);
template <typename R>
void adj_lens(const LensAdjArgs<R>& A, cudaStream_t st, Prof* pf);

// One cosmology of a lens dot product: chi tables (TabId), source distances,
// weight prefactor, the shell's D1(a_{i+1}) and g_p(a_{i+1/2}), accumulator.
struct LensDotVar {
  int tab_d1, tab_inva, qkind;  // TabIds, QKind of the n(z) tables
  const double* chi_s;
  double wpref, d1_next, gp_half;
  double* acc;
};
// lens kernel in "dot" mode for two cosmologies on the selection (shell bounds,
// replicas) of `sel`: a.acc += sum lam * (map increment under a), same for b
// (lam in the path precision)
template <typename R>
cudaError_t launch_lens_dot2(pm_ctx* c, const LensShell& sel, int use_pgd, const R* lam, const LensDotVar& a,
                             const LensDotVar& b);

// ---------------------------------------------------------- tangent-linear (jvp.cu)
// IC: dx, dp from the tangent displacements (lattice order)
template <typename R>
cudaError_t launch_tan_ic(pm_ctx* c, R* const* dpsi1, R* const* dpsi2, double d1, double d2, double g1, double g2);
// tangent of the 2LPT source from the base (d) and tangent (dd) second derivatives
template <typename R>
cudaError_t launch_lpt2_source_tan(pm_ctx* c, R* const* d, R* const* dd, R* out, long long n);
// d rho from dx at the current positions (rho zeroed by the caller)
template <typename R>
cudaError_t launch_tan_paint(pm_ctx* c, R* rho);
// tangent kick + drift of step i at x_i (F at fmesh_at(c), dF at L.tan_f)
template <typename R>
cudaError_t launch_tan_kd(pm_ctx* c, double ckick, double cdrift);
// tangent of a shell's map increments into L.tan_maps
template <typename R>
cudaError_t launch_tan_lens(pm_ctx* c, const LensShell& sh, int use_pgd);
// re-order the tangent state after a sort of the particle state
template <typename R>
cudaError_t tan_permute(pm_ctx* c, const uint32_t* old_pid, const uint32_t* new_pid);

}  // namespace pmlens
