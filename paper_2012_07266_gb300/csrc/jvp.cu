// Tangent-linear (forward-mode) kernels: the derivative of the forward model
// along a direction of the initial white noise (Sec. 3: the model is
// differentiable in the initial modes; the paper checks its Jacobian-vector
// product by changing the initial field in one pixel, Fig. 8).
//
// The tangent state (dx, dp in force-mesh cells, particle order of the primal
// state) is carried alongside the forward run:
//  * initial conditions: dPsi1 is linear in the noise; the 2LPT source
//    sum_{a<b} (phi_aa phi_bb - phi_ab^2) has the tangent
//    sum_{a<b} (dphi_aa phi_bb + phi_aa dphi_bb - 2 phi_ab dphi_ab);
//    dx = (D1 dPsi1 + D2 dPsi2) / cell, dp = (g_p dPsi1 + g_p2 dPsi2) / cell;
//  * force at x: d F(x) = grad(F mesh)(x) . dx + (force of d rho)(x), with
//    d rho = sum_j m dx_j . grad w_c(x_j) (the CIC weight gradients), painted
//    here and transformed by the same spectral force operator as rho;
//  * kick dp += kick_i dF(x_i), drift dx += drift_i dp;
//  * PGD: dS(x) = grad(S mesh)(x) . dx + (PGD field of d rho)(x);
//  * projection: selection and pixel fixed, the Born weight and the angular
//    CIC weights differentiated along the sub-evolved, displaced position.
#include <algorithm>
#include <cmath>

#include "adjoint.h"
#include "cic.cuh"
#include "lens_cull.cuh"

namespace pmlens {

namespace {

template <typename T>
__device__ __forceinline__ T pick3(int a, T v0, T v1, T v2) {
  return a == 0 ? v0 : (a == 1 ? v1 : v2);
}

__device__ __forceinline__ void unpack_cell(uint32_t c, int& ix, int& iy, int& iz) {
  ix = c & 1023u;
  iy = (c >> 10) & 1023u;
  iz = c >> 20;
}

template <typename R>
__device__ __forceinline__ R interp_tab(const R* __restrict__ t, int n, R hinv, R x) {
  const R u = x * hinv;
  int k = (int)u;
  if (k < 0) k = 0;
  if (k > n - 2) k = n - 2;
  const R f = u - (R)k;
  return t[k] * (R(1) - f) + t[k + 1] * f;
}

// CIC value and position gradient (per cell) of a mesh at the particle
template <typename R>
__device__ __forceinline__ R value_grad(const R* __restrict__ m, const Corners& c, R fx, R fy, R fz, R* g) {
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R m000 = m[c.r00 + c.x0], m001 = m[c.r00 + c.x1], m010 = m[c.r01 + c.x0], m011 = m[c.r01 + c.x1];
  const R m100 = m[c.r10 + c.x0], m101 = m[c.r10 + c.x1], m110 = m[c.r11 + c.x0], m111 = m[c.r11 + c.x1];
  // rows (z, y) interpolated in x, and their x differences
  const R a00 = gx * m000 + fx * m001, a01 = gx * m010 + fx * m011;
  const R a10 = gx * m100 + fx * m101, a11 = gx * m110 + fx * m111;
  g[0] = gz * (gy * (m001 - m000) + fy * (m011 - m010)) + fz * (gy * (m101 - m100) + fy * (m111 - m110));
  g[1] = gz * (a01 - a00) + fz * (a11 - a10);
  g[2] = gy * (a10 - a00) + fy * (a11 - a01);
  return gz * (gy * a00 + fy * a01) + fz * (gy * a10 + fy * a11);
}

template <typename R>
__device__ __forceinline__ void add_pair(R* row, int x0, int x1, R a, R b) {
  if constexpr (sizeof(R) == 4) {
    red_pair(row, x0, x1, a, b);
  } else {
    atomicAdd(row + x0, a);
    atomicAdd(row + x1, b);
  }
}

struct TanState {
  const uint32_t* cell;
  const void* frac;  // 3 x np of R
  const void* mom;
};

// d rho = m sum_a dx_a d w_c / d x_a, deposited on the 8 corners
template <typename R>
__global__ void __launch_bounds__(256) k_tan_paint(TanState s, const R* __restrict__ dx, R* __restrict__ rho, int M,
                                                   R mass, long long np) {
  const R* fr = reinterpret_cast<const R*>(s.frac);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    unpack_cell(s.cell[j], ix, iy, iz);
    const Corners c = corners(M, ix, iy, iz);
    const R fx = fr[j], fy = fr[j + np], fz = fr[j + 2 * np];
    const R tx = mass * dx[j], ty = mass * dx[j + np], tz = mass * dx[j + 2 * np];
    const R wx[2] = {R(1) - fx, fx}, wy[2] = {R(1) - fy, fy}, wz[2] = {R(1) - fz, fz};
    const unsigned rows[4] = {c.r00, c.r01, c.r10, c.r11};  // (dz, dy) = (0,0), (0,1), (1,0), (1,1)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const R sy = dy ? R(1) : R(-1), sz = dz ? R(1) : R(-1);
      const R yz = wy[dy] * wz[dz];
      // corner (x0 | x1): -/+ tx wy wz + ty wx sy wz + tz wx wy sz
      const R common = ty * sy * wz[dz] + tz * wy[dy] * sz;
      add_pair(rho + rows[q], c.x0, c.x1, -tx * yz + wx[0] * common, tx * yz + wx[1] * common);
    }
  }
}

// tangent kick and drift at x_i: dp += kick (dF-mesh(x) + grad F(x) . dx); dx += drift dp
template <typename R>
__global__ void __launch_bounds__(256) k_tan_kd(TanState s, const R* __restrict__ F0, const R* __restrict__ F1,
                                                const R* __restrict__ F2, const R* __restrict__ T0,
                                                const R* __restrict__ T1, const R* __restrict__ T2,
                                                R* __restrict__ dx, R* __restrict__ dp, int M, R ckick, R cdrift,
                                                long long np) {
  const R* fr = reinterpret_cast<const R*>(s.frac);
  const R* Fm[3] = {F0, F1, F2};
  const R* Tm[3] = {T0, T1, T2};
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    unpack_cell(s.cell[j], ix, iy, iz);
    const Corners c = corners(M, ix, iy, iz);
    const R fx = fr[j], fy = fr[j + np], fz = fr[j + 2 * np];
    const R d0 = dx[j], d1 = dx[j + np], d2 = dx[j + 2 * np];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      R g[3];
      value_grad(Fm[k], c, fx, fy, fz, g);
      const R dF = gather(Tm[k], c, fx, fy, fz) + g[0] * d0 + g[1] * d1 + g[2] * d2;
      const R np_ = dp[j + k * np] + ckick * dF;
      dp[j + k * np] = np_;
      dx[j + k * np] += cdrift * np_;
    }
  }
}

template <typename R>
__global__ void k_tan_ic(const R* __restrict__ a0, const R* __restrict__ a1, const R* __restrict__ a2,
                         const R* __restrict__ b0, const R* __restrict__ b1, const R* __restrict__ b2,
                         R* __restrict__ dx, R* __restrict__ dp, double cpl, double d1, double d2, double g1,
                         double g2, long long np) {
  const R* A[3] = {a0, a1, a2};
  const R* B[3] = {b0, b1, b2};
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double s1 = A[k][j], s2 = B[k] ? (double)B[k][j] : 0.0;
      dx[j + k * np] = (R)((d1 * s1 + d2 * s2) * cpl);
      dp[j + k * np] = (R)((g1 * s1 + g2 * s2) * cpl);
    }
  }
}

template <typename R>
__global__ void k_lpt2_source_tan(const R* __restrict__ d00, const R* __restrict__ d11, const R* __restrict__ d22,
                                  const R* __restrict__ d01, const R* __restrict__ d02, const R* __restrict__ d12,
                                  const R* __restrict__ e00, const R* __restrict__ e11, const R* __restrict__ e22,
                                  const R* __restrict__ e01, const R* __restrict__ e02, const R* __restrict__ e12,
                                  R* __restrict__ out, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const R a = d00[j], b = d11[j], c = d22[j], e = d01[j], f = d02[j], g = d12[j];
    const R da = e00[j], db = e11[j], dc = e22[j], de = e01[j], df = e02[j], dg = e12[j];
    out[j] = da * b + a * db + da * c + a * dc + db * c + b * dc - R(2) * (e * de + f * df + g * dg);
  }
}

template <typename R>
struct LensTanArgs {
  TanState st;
  const R *S0, *S1, *S2;     // PGD meshes (cells) or null
  const R *dS0, *dS1, *dS2;  // their tangents
  const R *dx, *dp;          // tangent state (cells)
  long long np;
  int M;
  double cell_len, chi_lo2, chi_hi2, fov_half, inv_dtheta, tan_half, margin;
  int npix, nzs, sub;
  double chi_s[PM_MAX_ZS];
  double wpref, d1_next, inv_gp_half, tab_hinv;
  R chi_s_r[PM_MAX_ZS], wpref_r, d1_next_r, inv_gp_half_r;  // the same rounded to R on the host
  GeomMirrors<R> g;                                          // the geometry scalars rounded to R
  int tab_n;
  const R *tab_d1, *tab_dd1, *tab_inva, *tab_dinva;
  unsigned nz_mask;       // bit s: source s is a distribution n(z)
  const R *qtab, *dqtab;  // its q(chi) and dq/dchi, n_zs x tab_n
  double* dmaps;
  int nrep;
  Replica rep[kMaxReplicas];
};

// Tangent of a shell's map increments: per (particle, live replica) in the shell,
// d(w cw_k) = dw/dchi_c dchi_c cw_k + w d cw_k, deposited on the same pixels.
template <typename R>
__global__ void __launch_bounds__(256) k_tan_lens(const LensTanArgs<R> A) {
  const R cell_len = A.g.cell_len;
  const R fov_half = A.g.fov_half, inv_dth = A.g.inv_dtheta;
  const R tan_half = A.g.tan_half, margin = A.g.margin;
  const R* fr = reinterpret_cast<const R*>(A.st.frac);
  const R* mo = reinterpret_cast<const R*>(A.st.mom);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); j0 < A.np; j0 += stride) {
    const bool valid = j0 + lane < A.np;
    const long long j = valid ? j0 + lane : A.np - 1;
    int ci0, ci1, ci2;
    unpack_cell(A.st.cell[j], ci0, ci1, ci2);
    const R cf0 = fr[j], cf1 = fr[j + A.np], cf2 = fr[j + 2 * A.np];
    const R cp0 = mo[j], cp1 = mo[j + A.np], cp2 = mo[j + 2 * A.np];
    const R tx0 = A.dx[j], tx1 = A.dx[j + A.np], tx2 = A.dx[j + 2 * A.np];
    const R tp0 = A.dp[j], tp1 = A.dp[j + A.np], tp2 = A.dp[j + 2 * A.np];
    R cs0 = R(0), cs1 = R(0), cs2 = R(0), ts0 = R(0), ts1 = R(0), ts2 = R(0);
    bool have_s = false;
    const WarpBox box = warp_box(valid, (float)ci0 + (float)cf0, (float)ci1 + (float)cf1, (float)ci2 + (float)cf2);
    // the particle's PGD displacement and its tangent (cells)
    auto gather_s = [&]() {
      const Corners cc = corners(A.M, ci0, ci1, ci2);
      const R* Sm[3] = {A.S0, A.S1, A.S2};
      const R* dSm[3] = {A.dS0, A.dS1, A.dS2};
      R sv[3], tv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        R g[3];
        sv[k] = value_grad(Sm[k], cc, cf0, cf1, cf2, g);
        tv[k] = gather(dSm[k], cc, cf0, cf1, cf2) + g[0] * tx0 + g[1] * tx1 + g[2] * tx2;
      }
      cs0 = sv[0]; cs1 = sv[1]; cs2 = sv[2];
      ts0 = tv[0]; ts1 = tv[1]; ts2 = tv[2];
      have_s = true;
    };
    auto project = [&](int q) {
      const Replica rp = A.rep[q];
      R r[3], pr[3], dr[3], dpr[3], gf[3];
      R sg[3];
      int gi[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int ax = rp.perm[d];
        int i = pick3(ax, ci0, ci1, ci2);
        R f = pick3(ax, cf0, cf1, cf2);
        sg[d] = R(1);
        if (rp.flip >> d & 1) {
          if (f > R(0)) { i = A.M - 1 - i; f = R(1) - f; }
          else { i = i == 0 ? 0 : A.M - i; }
          sg[d] = R(-1);
        }
        i += rp.shift[d];
        if (i >= A.M) i -= A.M;
        gi[d] = i + rp.n[d] * A.M;
        gf[d] = f;
        r[d] = ((R)gi[d] + f) * cell_len;
        pr[d] = sg[d] * pick3(ax, cp0, cp1, cp2);
        dr[d] = sg[d] * pick3(ax, tx0, tx1, tx2) * cell_len;
        dpr[d] = sg[d] * pick3(ax, tp0, tp1, tp2);
      }
      const R chi2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (!(r[2] > R(0) && in_shell<R>(chi2, gi, gf, A.cell_len, A.chi_lo2, A.chi_hi2, A.g.lo2, A.g.hi2))) return;
      const R lim = r[2] * tan_half + margin;
      if (fabs(r[0]) > lim || fabs(r[1]) > lim) return;
      if (A.S0 && !have_s) gather_s();
      R rc[3], drc[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) { rc[d] = r[d]; drc[d] = dr[d]; }
      if (A.sub) {
        const R chi = sqrt(chi2);
        const R t = interp_tab<R>(A.tab_d1, A.tab_n, A.g.tab_hinv, chi);
        const R dt = (t - A.d1_next_r) * A.inv_gp_half_r * cell_len;
        const R ddt = interp_tab<R>(A.tab_dd1, A.tab_n, A.g.tab_hinv, chi) * A.inv_gp_half_r * cell_len;
        const R dchi = (r[0] * dr[0] + r[1] * dr[1] + r[2] * dr[2]) / chi;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          rc[d] += pr[d] * dt;
          drc[d] += dpr[d] * dt + pr[d] * ddt * dchi;
        }
      }
      if (A.S0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int ax = rp.perm[d];
          rc[d] += sg[d] * pick3(ax, cs0, cs1, cs2) * cell_len;
          drc[d] += sg[d] * pick3(ax, ts0, ts1, ts2) * cell_len;
        }
      }
      if (!(rc[2] > R(0))) return;
      const R chic = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
      const R dchic = (rc[0] * drc[0] + rc[1] * drc[1] + rc[2] * drc[2]) / chic;
      const R inz = R(1) / rc[2];
      const R u = (rc[0] * inz + fov_half) * inv_dth - R(0.5);
      const R v = (rc[1] * inz + fov_half) * inv_dth - R(0.5);
      if (!isfinite(u) || !isfinite(v)) return;
      if (u < R(-1) || v < R(-1) || u >= (R)A.npix || v >= (R)A.npix) return;
      const R du = (drc[0] - rc[0] * inz * drc[2]) * inz * inv_dth;
      const R dv = (drc[1] - rc[1] * inz * drc[2]) * inz * inv_dth;
      const R fu0 = floor(u), fv0 = floor(v);
      const int iu = (int)fu0, iv = (int)fv0;
      const R fu = u - fu0, fv = v - fv0;
      const R inva = interp_tab<R>(A.tab_inva, A.tab_n, A.g.tab_hinv, chic);
      const R dinva = interp_tab<R>(A.tab_dinva, A.tab_n, A.g.tab_hinv, chic);
      for (int s = 0; s < A.nzs; ++s) {
        R w, dw;
        if (A.nz_mask >> s & 1u) {
          // source distribution: w = wpref q / (chi a)
          const R qv = interp_tab<R>(A.qtab + (size_t)s * A.tab_n, A.tab_n, A.g.tab_hinv, chic);
          if (!(qv > R(0))) continue;
          const R dqv = interp_tab<R>(A.dqtab + (size_t)s * A.tab_n, A.tab_n, A.g.tab_hinv, chic);
          w = A.wpref_r * qv / chic * inva;
          dw = A.wpref_r * ((dqv * chic - qv) / (chic * chic) * inva + qv / chic * dinva) * dchic;
        } else {
          const R csd = A.chi_s_r[s];
          if (!(chic < csd)) continue;
          const R fq = R(1) / chic - R(1) / csd;
          w = A.wpref_r * fq * inva;
          dw = A.wpref_r * (-inva / (chic * chic) + fq * dinva) * dchic;
        }
        const int off = s * A.npix * A.npix;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int ku = k & 1, kv = k >> 1;
          const int jx = iu + ku, jy = iv + kv;
          if (jx < 0 || jx >= A.npix || jy < 0 || jy >= A.npix) continue;
          const R wu = ku ? fu : R(1) - fu, wv = kv ? fv : R(1) - fv;
          const R dwu = ku ? du : -du, dwv = kv ? dv : -dv;
          atomicAdd(A.dmaps + off + jy * A.npix + jx, to_f64(dw * wu * wv + w * (dwu * wv + wu * dwv)));
        }
      }
    };
    for (int base = 0; base < A.nrep; base += 32) {
      // replicas base..base+31 any particle of the warp may reach (warp-uniform ballot)
      unsigned live = cull_replicas(A.rep, A.nrep, base, box, A.M, A.g.cull_cell_len, A.g.cull_lo2, A.g.cull_hi2,
                                    A.g.cull_tan_half, A.g.cull_margin);
      if (!valid) live = 0u;
      if (A.S0 && live && !have_s) gather_s();  // as in the forward: before the per-replica tests
      while (live) {
        const int q = base + __ffs(live) - 1;
        live &= live - 1u;
        project(q);
      }
    }
  }
}

TanState tan_state(pm_ctx* c) {
  TanState s;
  s.cell = reinterpret_cast<const uint32_t*>(c->ws + c->L.cell);
  s.frac = c->ws + c->L.frac;
  s.mom = c->ws + c->L.mom;
  return s;
}

int blocks_n(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152LL * 16); }

}  // namespace

template <typename R>
cudaError_t launch_tan_ic(pm_ctx* c, R* const* dpsi1, R* const* dpsi2, double d1, double d2, double g1, double g2) {
  ProfScope ps(&c->prof, KK_JVP, c->stream);
  R* dx = reinterpret_cast<R*>(c->ws + c->L.tan_x);
  R* dp = reinterpret_cast<R*>(c->ws + c->L.tan_p);
  const double cpl = c->M / c->cfg.box;
  k_tan_ic<R><<<blocks_n(c->np), 256, 0, c->stream>>>(dpsi1[0], dpsi1[1], dpsi1[2], dpsi2 ? dpsi2[0] : nullptr,
                                                      dpsi2 ? dpsi2[1] : nullptr, dpsi2 ? dpsi2[2] : nullptr, dx, dp,
                                                      cpl, d1, d2, g1, g2, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lpt2_source_tan(pm_ctx* c, R* const* d, R* const* dd, R* out, long long n) {
  ProfScope ps(&c->prof, KK_JVP, c->stream);
  k_lpt2_source_tan<R><<<blocks_n(n), 256, 0, c->stream>>>(d[0], d[1], d[2], d[3], d[4], d[5], dd[0], dd[1], dd[2],
                                                           dd[3], dd[4], dd[5], out, n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tan_paint(pm_ctx* c, R* rho) {
  const double mass = std::pow((double)c->M / c->nc, 3.0);
  ProfScope ps(&c->prof, KK_JVP, c->stream, c->np * (4.0 + 6.0 * sizeof(R)) + 2.0 * c->mesh_elems * sizeof(R));
  k_tan_paint<R><<<blocks_n(c->np), 256, 0, c->stream>>>(tan_state(c), reinterpret_cast<const R*>(c->ws + c->L.tan_x),
                                                         rho, c->M, (R)mass, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tan_kd(pm_ctx* c, double ckick, double cdrift) {
  const R* F = reinterpret_cast<const R*>(c->ws + fmesh_at(c));
  const R* T = reinterpret_cast<const R*>(c->ws + c->L.tan_f);
  const size_t m = c->mesh_elems;
  ProfScope ps(&c->prof, KK_JVP, c->stream, c->np * (4.0 + 15.0 * sizeof(R)) + 6.0 * m * sizeof(R));
  k_tan_kd<R><<<blocks_n(c->np), 256, 0, c->stream>>>(tan_state(c), F, F + m, F + 2 * m, T, T + m, T + 2 * m,
                                                      reinterpret_cast<R*>(c->ws + c->L.tan_x),
                                                      reinterpret_cast<R*>(c->ws + c->L.tan_p), c->M, (R)ckick,
                                                      (R)cdrift, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tan_lens(pm_ctx* c, const LensShell& sh, int use_pgd) {
  LensTanArgs<R> A;
  A.st = tan_state(c);
  const size_t m = c->mesh_elems;
  if (use_pgd) {
    const R* S = reinterpret_cast<const R*>(c->ws + smesh_at(c));
    const R* dS = reinterpret_cast<const R*>(c->ws + c->L.tan_s);
    A.S0 = S; A.S1 = S + m; A.S2 = S + 2 * m;
    A.dS0 = dS; A.dS1 = dS + m; A.dS2 = dS + 2 * m;
  } else {
    A.S0 = A.S1 = A.S2 = A.dS0 = A.dS1 = A.dS2 = nullptr;
  }
  A.dx = reinterpret_cast<const R*>(c->ws + c->L.tan_x);
  A.dp = reinterpret_cast<const R*>(c->ws + c->L.tan_p);
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
  A.sub = c->cfg.sub_evolution;
  for (int s = 0; s < PM_MAX_ZS; ++s) A.chi_s[s] = s < c->cfg.n_zs ? c->chi_s[s] : 0.0;
  const double vp = std::pow(c->cfg.box / c->nc, 3.0);
  A.wpref = 1.5 * c->cfg.omega_m / (kCoverH0 * kCoverH0) * vp / (dth * dth);
  A.d1_next = sh.d1_next;
  A.inv_gp_half = 1.0 / sh.gp_half;
  A.tab_hinv = 1.0 / c->chi_tab_h;
  for (int s = 0; s < PM_MAX_ZS; ++s) A.chi_s_r[s] = (R)A.chi_s[s];
  A.wpref_r = (R)A.wpref;
  A.d1_next_r = (R)A.d1_next;
  A.inv_gp_half_r = (R)A.inv_gp_half;
  A.g = geom_mirrors<R>(A.cell_len, A.chi_lo2, A.chi_hi2, A.fov_half, A.inv_dtheta, A.tan_half, A.margin,
                        A.tab_hinv);
  A.tab_n = kChiTab;
  A.tab_d1 = chi_table<R>(c, T_D1);
  A.tab_dd1 = chi_table<R>(c, T_DD1);
  A.tab_inva = chi_table<R>(c, T_INVA);
  A.tab_dinva = chi_table<R>(c, T_DINVA);
  A.nz_mask = c->nz_mask;
  A.qtab = qtable<R>(c, Q_CENTRAL);
  A.dqtab = qtable<R>(c, Q_DERIV);
  A.dmaps = reinterpret_cast<double*>(c->ws + c->L.tan_maps);
  A.nrep = sh.nrep;
  for (int q = 0; q < sh.nrep; ++q) A.rep[q] = sh.rep[q];
  ProfScope ps(&c->prof, KK_JVP, c->stream, c->np * (4.0 + 12.0 * sizeof(R)));
  k_tan_lens<R><<<(int)std::min<long long>((c->np + 255) / 256, 152LL * 8), 256, 0, c->stream>>>(A);
  return cudaGetLastError();
}

// after a re-sort of the state (old order old_pid, new order new_pid): the same
// permutation for the tangent state, through lattice order
template <typename R>
cudaError_t tan_permute(pm_ctx* c, const uint32_t* old_pid, const uint32_t* new_pid) {
  R* tmp = reinterpret_cast<R*>(c->ws + c->L.tan_tmp);
  for (size_t off : {c->L.tan_x, c->L.tan_p}) {
    R* a = reinterpret_cast<R*>(c->ws + off);
    if (cudaError_t e = launch_unpermute3<R>(c, a, old_pid, tmp)) return e;
    if (cudaError_t e = launch_permute3<R>(c, tmp, new_pid, a)) return e;
  }
  return cudaSuccess;
}

#define PM_JVP_INST(R)                                                                                       \
  template cudaError_t launch_tan_ic<R>(pm_ctx*, R* const*, R* const*, double, double, double, double);     \
  template cudaError_t launch_lpt2_source_tan<R>(pm_ctx*, R* const*, R* const*, R*, long long);             \
  template cudaError_t launch_tan_paint<R>(pm_ctx*, R*);                                                     \
  template cudaError_t launch_tan_kd<R>(pm_ctx*, double, double);                                            \
  template cudaError_t launch_tan_lens<R>(pm_ctx*, const LensShell&, int);                                   \
  template cudaError_t tan_permute<R>(pm_ctx*, const uint32_t*, const uint32_t*);
PM_JVP_INST(float)
PM_JVP_INST(double)

}  // namespace pmlens
