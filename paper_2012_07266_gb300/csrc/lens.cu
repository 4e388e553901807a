// Born lightcone projection (Eq. conv) with box replication/rotation and the
// sub-evolution scheme (Sec. 3), and the final mean-density subtraction.
//
// One thread per particle, replicas looped in registers: the particle is read
// once (cell, fraction, momentum, optional PGD displacement gathered from the
// PGD meshes) and tested against every replica the warp may reach.  Geometry
// and the lensing weights run in the path's precision (FP32 fast path:
// positions in Mpc/h to ~1e-7 relative; shell membership near a boundary
// decided in FP64), the map accumulation always in FP64.
#include <algorithm>
#include <cmath>

#include "adjoint.h"
#include "lens_cull.cuh"

namespace pmlens {

namespace {

// Cosmology-dependent part of a projection: growth and 1/a tables, source
// distances, weight prefactor, the shell's D1(a_{i+1}) and 1/g_p(a_{i+1/2}), and
// (dot mode) where the dot product accumulates.
template <typename R>
struct LensVar {
  const R* tab_d1;    // D1(a(chi)) on a uniform chi grid (path precision)
  const R* tab_inva;  // 1 / a(chi)
  double chi_s[PM_MAX_ZS];
  double wpref;       // (3/2) Om (H0/c)^2 V_p / Omega_pix
  double d1_next, inv_gp_half;
  R chi_s_r[PM_MAX_ZS], wpref_r, d1_next_r, inv_gp_half_r;  // the same rounded to R on the host
  const R* qtab;      // q(chi) of the n(z) sources, n_zs x tab_n (sources in nz_mask)
  double* acc;
};

template <typename R>
struct LensArgs {
  const uint32_t* cell;
  const R *fx, *fy, *fz, *px, *py, *pz;
  const R *S0, *S1, *S2;  // PGD displacement meshes (cells), or null
  long long np;
  int M;
  double cell_len;
  double chi_lo2, chi_hi2;
  double fov_half, inv_dtheta;
  double tan_half;  // tan of half the field of view plus one pixel
  double margin;    // bound on the sub-evolution + PGD displacement (Mpc/h)
  int npix, nzs, sub;
  double tab_hinv;
  int tab_n;
  LensVar<R> var[2];  // var[0]; dot mode may add a second cosmology (var[1]) on the same selection
  unsigned nz_mask;   // bit s: source s is a distribution n(z) (weight from var.qtab)
  double* maps;
  int* flag;
  unsigned long long* gathers;  // count of PGD gathers (forward projection), or null
  const R* lam;       // when set: accumulate sum(lam * increment) into var[v].acc instead of the maps
  GeomMirrors<R> g;   // the geometry scalars above rounded to R (and FP32 for the culling)
  int nrep;
  Replica rep[kMaxReplicas];
};

struct MeanTerms { double v[PM_MAX_ZS]; };

// block-wide sum of one double into *acc
__device__ __forceinline__ void block_sum(double v, double* acc) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(acc, v);
  }
}

template <typename T>
__device__ __forceinline__ T pick3(int a, T v0, T v1, T v2) {
  return a == 0 ? v0 : (a == 1 ? v1 : v2);
}

template <typename R>
__device__ __forceinline__ R interp(const R* __restrict__ t, int n, R hinv, R x) {
  const R u = x * hinv;
  int k = (int)u;
  if (k < 0) k = 0;
  if (k > n - 2) k = n - 2;
  const R f = u - (R)k;
  return t[k] * (R(1) - f) + t[k + 1] * f;
}

template <typename R>
__device__ __forceinline__ R gather3(const R* __restrict__ m, int M, int ix, int iy, int iz, R fx, R fy, R fz) {
  const int ix1 = ix + 1 == M ? 0 : ix + 1, iy1 = iy + 1 == M ? 0 : iy + 1, iz1 = iz + 1 == M ? 0 : iz + 1;
  const long long r00 = ((long long)iz * M + iy) * M, r01 = ((long long)iz * M + iy1) * M;
  const long long r10 = ((long long)iz1 * M + iy) * M, r11 = ((long long)iz1 * M + iy1) * M;
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R a = gx * m[r00 + ix] + fx * m[r00 + ix1];
  const R b = gx * m[r01 + ix] + fx * m[r01 + ix1];
  const R d = gx * m[r10 + ix] + fx * m[r10 + ix1];
  const R e = gx * m[r11 + ix] + fx * m[r11 + ix1];
  return gz * (gy * a + fy * b) + fz * (gy * d + fy * e);
}

// Geometry runs in the path's precision R (FP32 fast path, FP64 plain path).
// NV cosmology variants share the particle read, the replica transform, the
// shell selection and the PGD gather (NV = 2: the Omega_m +/- h dot products).
template <typename R, int NV>
__global__ void __launch_bounds__(256) k_lens(const LensArgs<R> A) {
  const R cell_len = A.g.cell_len;
  const R fov_half = A.g.fov_half, inv_dth = A.g.inv_dtheta;
  const R tan_half = A.g.tan_half, margin = A.g.margin;
  R dot[NV];
#pragma unroll
  for (int vi = 0; vi < NV; ++vi) dot[vi] = R(0);
  unsigned ngath = 0;  // particles of this thread whose PGD displacement was gathered
  // whole warps iterate together (warp-level replica culling); lanes past the end add nothing
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); j0 < A.np; j0 += stride) {
    const bool valid = j0 + lane < A.np;
    const long long j = valid ? j0 + lane : A.np - 1;
    const uint32_t c = A.cell[j];
    // per-axis particle data in registers; a replica's axis permutation picks
    // among them with selects (a runtime-indexed array would live in local memory)
    const int ci0 = (int)(c & 1023u), ci1 = (int)((c >> 10) & 1023u), ci2 = (int)(c >> 20);
    const R cf0 = A.fx[j], cf1 = A.fy[j], cf2 = A.fz[j];
    const R cp0 = A.px[j], cp1 = A.py[j], cp2 = A.pz[j];
    R cs0 = R(0), cs1 = R(0), cs2 = R(0);
    bool have_s = false;  // PGD displacement gathered only for particles that may land on the map
    const WarpBox box = warp_box(valid, (float)ci0 + (float)cf0, (float)ci1 + (float)cf1, (float)ci2 + (float)cf2);
    // one replica of this particle (the per-particle tests below decide exactly)
    auto project = [&](int q) {
      const Replica rp = A.rep[q];
      R r[3], pr[3], sr[3], gf[3];
      int gi[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int ax = rp.perm[d];
        int i = pick3(ax, ci0, ci1, ci2);
        R f = pick3(ax, cf0, cf1, cf2);
        R sg = R(1);
        if (rp.flip >> d & 1) {
          if (f > R(0)) { i = A.M - 1 - i; f = R(1) - f; }
          else { i = i == 0 ? 0 : A.M - i; }
          sg = R(-1);
        }
        i += rp.shift[d];
        if (i >= A.M) i -= A.M;
        gi[d] = i + rp.n[d] * A.M;
        gf[d] = f;
        r[d] = ((R)gi[d] + f) * cell_len;
        pr[d] = sg * pick3(ax, cp0, cp1, cp2);
        sr[d] = sg * pick3(ax, cs0, cs1, cs2);
      }
      const R chi2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (!(r[2] > R(0) && in_shell<R>(chi2, gi, gf, A.cell_len, A.chi_lo2, A.chi_hi2, A.g.lo2, A.g.hi2))) return;
      // outside the field of view by more than the displacement margin: no weight on the map
      const R lim = r[2] * tan_half + margin;
      if (fabs(r[0]) > lim || fabs(r[1]) > lim) return;
      if (A.S0 && !have_s) {
        cs0 = gather3(A.S0, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        cs1 = gather3(A.S1, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        cs2 = gather3(A.S2, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        have_s = true;
        ++ngath;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const R v = pick3((int)rp.perm[d], cs0, cs1, cs2);
          sr[d] = (rp.flip >> d & 1) ? -v : v;
        }
      }
      const R chi = A.sub ? sqrt(chi2) : R(0);
#pragma unroll
      for (int vi = 0; vi < NV; ++vi) {
        const LensVar<R>& V = A.var[vi];
        R q[3] = {r[0], r[1], r[2]};
        if (A.sub) {
          const R t = interp<R>(V.tab_d1, A.tab_n, A.g.tab_hinv, chi);
          const R dt = (t - V.d1_next_r) * V.inv_gp_half_r * cell_len;
#pragma unroll
          for (int d = 0; d < 3; ++d) q[d] += pr[d] * dt;
        }
        if (A.S0) {
#pragma unroll
          for (int d = 0; d < 3; ++d) q[d] += sr[d] * cell_len;
        }
        if (!(q[2] > R(0))) continue;
        const R chic = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        const R inz = R(1) / q[2];
        const R u = (q[0] * inz + fov_half) * inv_dth - R(0.5);
        const R v = (q[1] * inz + fov_half) * inv_dth - R(0.5);
        if (!isfinite(u) || !isfinite(v) || !isfinite(chic)) {
          atomicOr(A.flag, 1);
          continue;
        }
        if (u < R(-1) || v < R(-1) || u >= (R)A.npix || v >= (R)A.npix) continue;
        const R fu0 = floor(u), fv0 = floor(v);
        const int iu = (int)fu0, iv = (int)fv0;
        const R fu = u - fu0, fv = v - fv0;
        // Born weight in the path's precision, map accumulation in FP64
        const R inva = interp<R>(V.tab_inva, A.tab_n, A.g.tab_hinv, chic);
        const R cw[4] = {(R(1) - fu) * (R(1) - fv), fu * (R(1) - fv), (R(1) - fu) * fv, fu * fv};
        const R wk = V.wpref_r * inva / chic;
        for (int s = 0; s < A.nzs; ++s) {
          R w;
          if (A.nz_mask >> s & 1u) {  // source distribution: w = wpref q(chi_c) / (chi_c a)
            const R qv = interp<R>(V.qtab + (size_t)s * A.tab_n, A.tab_n, A.g.tab_hinv, chic);
            if (!(qv > R(0))) continue;
            w = wk * qv;
          } else {  // source plane at chi_s
            const R cs_ = V.chi_s_r[s];
            if (!(chic < cs_)) continue;
            w = wk * (cs_ - chic) / cs_;
          }
          const int off = s * A.npix * A.npix;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int jx = iu + (k & 1), jy = iv + (k >> 1);
            if (jx >= 0 && jx < A.npix && jy >= 0 && jy < A.npix) {
              const int pix = off + jy * A.npix + jx;
              if (A.lam) dot[vi] += A.lam[pix] * w * cw[k];
              else atomicAdd(A.maps + pix, to_f64(w * cw[k]));
            }
          }
        }
      }
    };
    for (int base = 0; base < A.nrep; base += 32) {
      // replicas base..base+31 any particle of the warp may reach (warp-uniform ballot)
      unsigned live = cull_replicas(A.rep, A.nrep, base, box, A.M, A.g.cull_cell_len, A.g.cull_lo2, A.g.cull_hi2,
                                    A.g.cull_tan_half, A.g.cull_margin);
      if (!valid) live = 0u;
      // the PGD displacement of every particle of a warp that may reach the map, gathered
      // before the per-replica tests (which then find it in registers): its load latency
      // overlaps the replica geometry (0.528 -> 0.491 ms per pm256 launch)
      if (A.S0 && live && !have_s) {
        cs0 = gather3(A.S0, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        cs1 = gather3(A.S1, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        cs2 = gather3(A.S2, A.M, ci0, ci1, ci2, cf0, cf1, cf2);
        have_s = true;
        ++ngath;
      }
      while (live) {
        const int q = base + __ffs(live) - 1;
        live &= live - 1u;
        project(q);
      }
    }
  }
  if (A.gathers) {  // the particle loop is warp-uniform: every lane arrives here
    const unsigned t = __reduce_add_sync(0xffffffffu, ngath);
    if (lane == 0 && t) atomicAdd(A.gathers, (unsigned long long)t);
  }
  if (A.lam) {
#pragma unroll
    for (int vi = 0; vi < NV; ++vi) {
      if (vi) __syncthreads();  // block_sum's shared scratch is reused
      block_sum((double)dot[vi], A.var[vi].acc);
    }
  }
}

__global__ void k_kappa_finalize(const double* __restrict__ maps, double* __restrict__ out, long long npix2, int nzs,
                                 MeanTerms mt, int* flag) {
  const long long n = npix2 * nzs;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const double v = maps[j] - mt.v[j / npix2];
    if (!isfinite(v)) atomicOr(flag, 2);
    out[j] = v;
  }
}

}  // namespace

template <typename R>
static void fill_lens_args(pm_ctx* c, const LensShell& sh, int use_pgd, LensArgs<R>& A);

template <typename R>
static void var_mirrors(LensVar<R>& V) {
  for (int s = 0; s < PM_MAX_ZS; ++s) V.chi_s_r[s] = (R)V.chi_s[s];
  V.wpref_r = (R)V.wpref;
  V.d1_next_r = (R)V.d1_next;
  V.inv_gp_half_r = (R)V.inv_gp_half;
}

template <typename R>
cudaError_t launch_lens(pm_ctx* c, const LensShell& sh, int use_pgd) {
  LensArgs<R> A;
  fill_lens_args<R>(c, sh, use_pgd, A);
  long long blocks = (c->np + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  // particle state read once; the PGD gathers (mesh bytes in proportion to the particles
  // that gathered, counted on the device) are booked when the profile is read
  A.gathers = use_pgd ? lens_gather_count(c) : nullptr;
  ProfScope ps(&c->prof, KK_LENS, c->stream, c->np * (4.0 + 6.0 * sizeof(R)));
  k_lens<R, 1><<<(int)blocks, 256, 0, c->stream>>>(A);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lens_dot2(pm_ctx* c, const LensShell& sel, int use_pgd, const R* lam, const LensDotVar& a,
                             const LensDotVar& b) {
  LensArgs<R> A;
  fill_lens_args<R>(c, sel, use_pgd, A);
  const LensDotVar* in[2] = {&a, &b};
  for (int v = 0; v < 2; ++v) {
    LensVar<R>& V = A.var[v];
    V.tab_d1 = chi_table<R>(c, in[v]->tab_d1);
    V.tab_inva = chi_table<R>(c, in[v]->tab_inva);
    for (int s = 0; s < PM_MAX_ZS; ++s) V.chi_s[s] = s < c->cfg.n_zs ? in[v]->chi_s[s] : 0.0;
    V.wpref = in[v]->wpref;
    V.qtab = qtable<R>(c, in[v]->qkind);
    V.d1_next = in[v]->d1_next;
    V.inv_gp_half = 1.0 / in[v]->gp_half;
    V.acc = in[v]->acc;
    var_mirrors(V);
  }
  A.lam = lam;
  long long blocks = (c->np + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  ProfScope ps(&c->prof, KK_ADJ_LENS, c->stream, c->np * (4.0 + 6.0 * sizeof(R)));
  k_lens<R, 2><<<(int)blocks, 256, 0, c->stream>>>(A);
  return cudaGetLastError();
}

template <typename R>
static void fill_lens_args(pm_ctx* c, const LensShell& sh, int use_pgd, LensArgs<R>& A) {
  A.cell = reinterpret_cast<const uint32_t*>(c->ws + c->L.cell);
  const R* f = reinterpret_cast<const R*>(c->ws + c->L.frac);
  const R* p = reinterpret_cast<const R*>(c->ws + c->L.mom);
  A.fx = f; A.fy = f + c->np; A.fz = f + 2 * c->np;
  A.px = p; A.py = p + c->np; A.pz = p + 2 * c->np;
  if (use_pgd) {
    // the context's PGD meshes, or an adjoint segment slot
    const R* S = reinterpret_cast<const R*>(c->ws + smesh_at(c));
    A.S0 = S; A.S1 = S + c->mesh_elems; A.S2 = S + 2 * c->mesh_elems;
  } else {
    A.S0 = A.S1 = A.S2 = nullptr;
  }
  A.np = c->np;
  A.M = c->M;
  A.cell_len = c->cfg.box / c->M;
  A.chi_lo2 = sh.chi_lo2;
  A.chi_hi2 = sh.chi_hi2;
  const double fov = c->cfg.map_fov_deg * M_PI / 180.0;
  const double dth = fov / c->cfg.map_npix;
  A.fov_half = 0.5 * fov;
  A.inv_dtheta = 1.0 / dth;
  A.tan_half = std::tan(0.5 * fov + dth);
  A.margin = std::max(0.1 * c->cfg.box, 10.0);
  A.npix = c->cfg.map_npix;
  A.nzs = c->cfg.n_zs;
  LensVar<R>& V = A.var[0];
  for (int s = 0; s < PM_MAX_ZS; ++s) V.chi_s[s] = s < c->cfg.n_zs ? c->chi_s[s] : 0.0;
  const double vp = std::pow(c->cfg.box / c->nc, 3.0);
  V.wpref = 1.5 * c->cfg.omega_m / (kCoverH0 * kCoverH0) * vp / (dth * dth);
  V.d1_next = sh.d1_next;
  V.inv_gp_half = 1.0 / sh.gp_half;
  V.tab_d1 = chi_table<R>(c, T_D1);
  V.tab_inva = chi_table<R>(c, T_INVA);
  V.qtab = qtable<R>(c, Q_CENTRAL);
  V.acc = nullptr;
  var_mirrors(V);
  A.var[1] = V;
  A.sub = c->cfg.sub_evolution;
  A.tab_hinv = 1.0 / c->chi_tab_h;
  A.tab_n = kChiTab;
  A.maps = reinterpret_cast<double*>(c->ws + c->L.maps);
  A.flag = flags_ptr(c);
  A.gathers = nullptr;
  A.nz_mask = c->nz_mask;
  A.lam = nullptr;
  A.g = geom_mirrors<R>(A.cell_len, A.chi_lo2, A.chi_hi2, A.fov_half, A.inv_dtheta, A.tan_half, A.margin,
                        A.tab_hinv);
  A.nrep = sh.nrep;
  for (int q = 0; q < sh.nrep; ++q) A.rep[q] = sh.rep[q];
}

cudaError_t launch_kappa_finalize(pm_ctx* c, double* out) {
  const long long npix2 = (long long)c->cfg.map_npix * c->cfg.map_npix;
  MeanTerms mt;
  for (int s = 0; s < PM_MAX_ZS; ++s) mt.v[s] = s < c->cfg.n_zs ? c->mean_term[s] : 0.0;
  long long blocks = (npix2 * c->cfg.n_zs + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  ProfScope ps(&c->prof, KK_MISC, c->stream);
  k_kappa_finalize<<<(int)blocks, 256, 0, c->stream>>>(reinterpret_cast<const double*>(c->ws + c->L.maps), out,
                                                       npix2, c->cfg.n_zs, mt, flags_ptr(c));
  return cudaGetLastError();
}

template cudaError_t launch_lens<float>(pm_ctx*, const LensShell&, int);
template cudaError_t launch_lens<double>(pm_ctx*, const LensShell&, int);
template cudaError_t launch_lens_dot2<float>(pm_ctx*, const LensShell&, int, const float*, const LensDotVar&,
                                             const LensDotVar&);
template cudaError_t launch_lens_dot2<double>(pm_ctx*, const LensShell&, int, const double*, const LensDotVar&,
                                              const LensDotVar&);

}  // namespace pmlens
