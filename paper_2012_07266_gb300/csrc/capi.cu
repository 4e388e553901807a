// C ABI of the PM lensing library: context, workspace layout, host FP64
// tables, and the sequencing of the device work of each entry point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>

#include "adjoint.h"

using namespace pmlens;

namespace {

size_t al(size_t x) { return (x + 255) & ~size_t(255); }
int round16(int x) { return (x + 15) / 16 * 16; }

pm_status check_config(const pm_config* c) {
  if (!c) return PM_ERR_ARG;
  if (c->nc < 2 || c->nmesh < 2 || c->nmesh > 1024 || c->nc > c->nmesh) return PM_ERR_ARG;
  if (!fft_supported(c->nmesh) || !fft_supported(c->nc)) return PM_ERR_UNSUPPORTED;
  if (!(c->box > 0) || !(c->omega_m > 0 && c->omega_m <= 1) || !(c->sigma8 > 0)) return PM_ERR_ARG;
  if (!(c->h > 0) || !(c->omega_b > 0 && c->omega_b < c->omega_m) || !(c->t_cmb > 0)) return PM_ERR_ARG;
  if (!(c->a_init > 1e-3 && c->a_init < 1) || c->nsteps < 1 || c->nsteps > 100000) return PM_ERR_ARG;
  if (c->lpt_order != 1 && c->lpt_order != 2) return PM_ERR_ARG;
  if (c->n_zs < 1 || c->n_zs > PM_MAX_ZS) return PM_ERR_ARG;
  for (int s = 0; s < c->n_zs; ++s)
    if (!(c->zs[s] > 0 && c->zs[s] < 1.0 / c->a_init - 1.0)) return PM_ERR_ARG;
  if (c->map_npix < 1 || c->map_npix > 16384 || !(c->map_fov_deg > 0 && c->map_fov_deg < 60)) return PM_ERR_ARG;
  if (c->precision != PM_FP32 && c->precision != PM_FP64) return PM_ERR_ARG;
  if (c->pgd && !(c->pgd_params[2] >= 0 && c->pgd_params[3] > 0 && c->pgd_params[4] > 0)) return PM_ERR_ARG;
  if (c->ckpt_every < 0) return PM_ERR_ARG;
  if (c->jvp != 0 && c->jvp != 1) return PM_ERR_ARG;
  return PM_OK;
}

void plan_layout(const pm_config& cfg, Layout& L, int& P, int& Pc) {
  const size_t rs = cfg.precision == PM_FP64 ? 8 : 4, cs = 2 * rs;
  const size_t M = cfg.nmesh, nc = cfg.nc, np = nc * nc * nc;
  P = round16((int)M / 2 + 1);
  Pc = round16((int)nc / 2 + 1);
  const size_t mesh = M * M * M * rs, cmesh = M * M * (size_t)P * cs;
  const size_t grid = np * rs, cgrid = nc * nc * (size_t)Pc * cs;
  size_t o = 0;
  L.cell = o; o += al(np * 4);
  L.frac = o; o += al(3 * np * rs);
  L.mom = o; o += al(3 * np * rs);
  L.pid = o; o += al(np * 4);
  L.cell2 = o; o += al(np * 4);
  L.frac2 = o; o += al(3 * np * rs);
  L.mom2 = o; o += al(3 * np * rs);
  L.pid2 = o; o += al(np * 4);
  L.sort_cnt = o; o += al(sort_scratch_bytes((int)M));
  L.fmesh = o; o += al(3 * mesh);
  L.smesh = o; o += cfg.pgd ? al(3 * mesh) : 0;
  L.maps = o; o += al((size_t)cfg.n_zs * cfg.map_npix * cfg.map_npix * 8);
  L.flags = o; o += 256;
  L.sqrtp = o; o += al((3 * (nc / 2) * (nc / 2) + 1) * 8);
  L.tab_d1 = o; o += al(kChiTab * 8);
  L.tab_inva = o; o += al(kChiTab * 8);
  L.ftab = o; o += T_COUNT * al(kChiTab * 4);
  L.qtab = o; o += al((size_t)4 * cfg.n_zs * kChiTab * 8);    // n(z) sources: q, dq, q(+h), q(-h)
  L.qtab_f = o; o += al((size_t)4 * cfg.n_zs * kChiTab * 4);
  L.scratch = o;
  const int nout = cfg.pgd ? 6 : 3;
  L.rho = o;
  L.cbuf = L.rho + al(mesh);
  L.ubuf = L.cbuf + al(cmesh);
  const size_t step_end = L.ubuf + nout * al(cmesh);
  L.ic_real = o;
  L.ic_cbuf = L.ic_real + al(grid);
  L.ic_u = L.ic_cbuf + al(cgrid);
  L.ic_out = L.ic_u + 9 * al(cgrid);
  const size_t ic_end = L.ic_out + 13 * al(grid);
  L.adj = std::max(step_end, ic_end);
  L.total = L.adj;
  L.state_bytes = 2 * al(np * 4) + 2 * al(3 * np * rs);  // cell | frac | mom | pid
  L.nck = 0;
  L.nic = 0;
  size_t a = L.adj;
  if (cfg.ckpt_every > 0 || cfg.jvp) {
    // derivative tables: dD1/dchi, d(1/a)/dchi and the Omega_m +/- h coefficient sets
    L.tab_dd1 = a; a += al(kChiTab * 8);
    L.tab_dinva = a; a += al(kChiTab * 8);
    L.tab_d1p = a; a += al(kChiTab * 8);
    L.tab_d1m = a; a += al(kChiTab * 8);
    L.tab_invap = a; a += al(kChiTab * 8);
    L.tab_invam = a; a += al(kChiTab * 8);
    L.sqrtp_p = a; a += al((3 * (nc / 2) * (nc / 2) + 1) * 8);
    L.sqrtp_m = a; a += al((3 * (nc / 2) * (nc / 2) + 1) * 8);
  }
  if (cfg.ckpt_every > 0) {
    const int k = cfg.ckpt_every;
    L.nck = (cfg.nsteps + k - 1) / k;
    L.nic = 28;
    L.adj_noise = a; a += al(grid);
    L.adj_ckpt = a; a += (size_t)L.nck * L.state_bytes;
    L.adj_seg = a; a += (size_t)(std::min(k, cfg.nsteps) + 1) * L.state_bytes;
    L.adj_fseg = a; a += (size_t)(std::min(k, cfg.nsteps) + 1) * 3 * al(mesh);  // force meshes of the segment
    // PGD meshes S(x_{i+1}) of the segment's lens steps, from the recompute
    L.adj_sseg = a; a += cfg.pgd ? (size_t)std::min(k, cfg.nsteps) * 3 * al(mesh) : 0;
    L.adj_lx = a; a += al(3 * np * rs);
    L.adj_lp = a; a += al(3 * np * rs);
    L.adj_v = a; a += al(3 * np * rs);
    L.adj_vs = a; a += al(3 * np * rs);
    L.adj_paint = a; a += 4 * al(mesh);  // three cotangent meshes, or (FP32) one float4-interleaved mesh
    L.adj_ic = a; a += (size_t)L.nic * al(grid);
    L.adj_lam = a; a += rs == 4 ? al((size_t)cfg.n_zs * cfg.map_npix * cfg.map_npix * 4) : 0;
    L.adj_acc = a; a += al((size_t)(4 * cfg.nsteps + 64) * 8);
  }
  if (cfg.jvp) {
    // tangent state along a noise direction: dx, dp (cells), a permutation buffer,
    // dF (and dS) meshes at the current positions, the tangent maps, IC fields
    L.tan_x = a; a += al(3 * np * rs);
    L.tan_p = a; a += al(3 * np * rs);
    L.tan_tmp = a; a += al(3 * np * rs);
    L.tan_f = a; a += 3 * al(mesh);
    L.tan_s = a; a += cfg.pgd ? 3 * al(mesh) : 0;
    L.tan_maps = a; a += al((size_t)cfg.n_zs * cfg.map_npix * cfg.map_npix * 8);
    L.tan_ic = a; a += 14 * al(grid);  // noise direction, 9 LPT fields, source, 3 Psi2
  }
  L.total = a;
}

template <typename R>
R* rp(pm_ctx* c, size_t off) { return reinterpret_cast<R*>(c->ws + off); }

size_t seg_off(pm_ctx* c, int j);
size_t fseg_off(pm_ctx* c, int j);
size_t sseg_off(pm_ctx* c, int j);

size_t cmesh_bytes(pm_ctx* c) { return (size_t)c->M * c->M * c->P * 2 * c->rsz; }
size_t cgrid_bytes(pm_ctx* c) { return (size_t)c->nc * c->nc * c->Pc * 2 * c->rsz; }

pm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PM_OK : PM_ERR_CUDA; }

// ------------------------------------------------------------ host tables
void build_tables(pm_ctx* c) {
  const pm_config& cfg = c->cfg;
  Cosmo& co = c->cosmo;
  co.init(cfg.omega_m, cfg.sigma8, cfg.h, cfg.n_s, cfg.omega_b, cfg.t_cmb);
  const int n = cfg.nsteps;
  c->a.resize(n + 1);
  c->ah.resize(n);
  for (int i = 0; i <= n; ++i) c->a[i] = cfg.a_init + (1.0 - cfg.a_init) * i / n;
  for (int i = 0; i < n; ++i) c->ah[i] = 0.5 * (c->a[i] + c->a[i + 1]);
  c->kick.resize(n);
  c->drift.resize(n);
  for (int i = 0; i < n; ++i) {
    const double aprev = i == 0 ? c->a[0] : c->ah[i - 1];
    c->kick[i] = (co.gp(c->ah[i]) - co.gp(aprev)) / co.gf(c->a[i]);
    c->drift[i] = (co.D1(c->a[i + 1]) - co.D1(c->a[i])) / co.gp(c->ah[i]);
  }
  c->chi_a.resize(n + 1);
  for (int i = 0; i <= n; ++i) c->chi_a[i] = co.chi_a(c->a[i]);
  c->chi_s.resize(cfg.n_zs);
  double chi_s_max = 0;
  for (int s = 0; s < cfg.n_zs; ++s) {
    c->chi_s[s] = co.chi_a(1.0 / (1.0 + cfg.zs[s]));
    chi_s_max = std::max(chi_s_max, c->chi_s[s]);
  }
  c->chi_tab_max = 1.1 * std::max(c->chi_a[0], chi_s_max) + 50.0;
  c->chi_tab_h = c->chi_tab_max / (kChiTab - 1);
  // mean-density term: (3/2) Om (H0/c)^2 int_0^chi_s chi (chi_s - chi) / (chi_s a) dchi (Simpson)
  for (int s = 0; s < PM_MAX_ZS; ++s) c->mean_term[s] = 0.0;
  std::vector<double> ag(8001);
  for (int s = 0; s < cfg.n_zs; ++s) {
    const double cs = c->chi_s[s];
    const int m = 8000;
    const double hh = cs / m;
    co.a_of_chi_grid(hh, m + 1, ag.data());
    double acc = 0;
    for (int k = 0; k <= m; ++k) {
      const double x = k * hh;
      const double f = x * (cs - x) / (cs * ag[k]);
      acc += (k == 0 || k == m ? 1.0 : (k & 1 ? 4.0 : 2.0)) * f;
    }
    c->mean_term[s] = 1.5 * cfg.omega_m / (kCoverH0 * kCoverH0) * acc * hh / 3.0;
  }
}

// ------------------------------------------------------ source distributions
// Lensing efficiency of a normalised, piecewise-linear n(z) (Eq. conv with a
// distribution of source distances) on the chi grid of the lens tables:
//   q(chi) = int dz' n(z') (1 - chi / chi(z'))_+ = A(chi) - chi B(chi),
//   A = int_{z(chi)} n dz',  B = int_{z(chi)} n / chi(z') dz',  dq/dchi = -B,
// with A and B cumulative trapezoid integrals from the top on a 20001-point
// redshift grid.  Returns the farthest contributing distance in chimax.
void nz_tables(const pm_ctx* c, const Cosmo& co, const std::vector<double>& z, const std::vector<double>& n,
               std::vector<double>& q, std::vector<double>& dq, double& chimax) {
  const int G = 20001;
  std::vector<double> zz(G), nn(G), ch(G), A(G), B(G);
  const double z0 = z.front(), z1 = z.back();
  size_t seg = 0;
  for (int k = 0; k < G; ++k) {
    zz[k] = z0 + (z1 - z0) * k / (G - 1);
    while (seg + 2 < z.size() && z[seg + 1] < zz[k]) ++seg;
    const double t = std::min(std::max((zz[k] - z[seg]) / (z[seg + 1] - z[seg]), 0.0), 1.0);
    nn[k] = n[seg] + t * (n[seg + 1] - n[seg]);
    ch[k] = co.chi_a(1.0 / (1.0 + zz[k]));
  }
  double norm = 0.0;
  for (int k = 0; k + 1 < G; ++k) norm += 0.5 * (nn[k] + nn[k + 1]) * (zz[k + 1] - zz[k]);
  A[G - 1] = B[G - 1] = 0.0;
  for (int k = G - 2; k >= 0; --k) {
    const double dz = zz[k + 1] - zz[k];
    A[k] = A[k + 1] + 0.5 * (nn[k] + nn[k + 1]) * dz / norm;
    B[k] = B[k + 1] + 0.5 * (nn[k] / ch[k] + nn[k + 1] / ch[k + 1]) * dz / norm;
  }
  chimax = ch[G - 1];
  q.assign(kChiTab, 0.0);
  dq.assign(kChiTab, 0.0);
  int j = 0;
  for (int k = 0; k < kChiTab; ++k) {
    const double x = k * c->chi_tab_h;
    double a = 0.0, b = 0.0;
    if (x <= ch[0]) {
      a = A[0];
      b = B[0];
    } else if (x < ch[G - 1]) {
      while (ch[j + 1] < x) ++j;
      const double t = (x - ch[j]) / (ch[j + 1] - ch[j]);
      a = A[j] + t * (A[j + 1] - A[j]);
      b = B[j] + t * (B[j + 1] - B[j]);
    }
    q[k] = std::max(a - x * b, 0.0);
    dq[k] = -b;
  }
}

// (3/2) Om (H0/c)^2 int_0^chimax chi q(chi) / a(chi) dchi on the table grid (trapezoid)
double nz_mean_term(const pm_ctx* c, const Cosmo& co, double om, const std::vector<double>& q) {
  std::vector<double> ag(kChiTab);
  co.a_of_chi_grid(c->chi_tab_h, kChiTab, ag.data());
  double acc = 0.0;
  for (int k = 0; k + 1 < kChiTab; ++k) {
    const double x0 = k * c->chi_tab_h, x1 = (k + 1) * c->chi_tab_h;
    acc += 0.5 * (x0 * q[k] / ag[k] + x1 * q[k + 1] / ag[k + 1]) * c->chi_tab_h;
  }
  return 1.5 * om / (kCoverH0 * kCoverH0) * acc;
}

// build and upload source s's tables (central cosmology, and the Omega_m +/- h
// pair when the derivative tables exist); the source's distance becomes chimax
cudaError_t set_nz_tables(pm_ctx* c, int s) {
  const pm_config& cfg = c->cfg;
  const bool deriv = cfg.ckpt_every > 0 || cfg.jvp;
  std::vector<double> tab[4];
  double chimax = 0.0, chip = 0.0, chim = 0.0;
  nz_tables(c, c->cosmo, c->nz_z[s], c->nz_n[s], tab[Q_CENTRAL], tab[Q_DERIV], chimax);
  c->chi_s[s] = chimax;
  c->mean_term[s] = nz_mean_term(c, c->cosmo, cfg.omega_m, tab[Q_CENTRAL]);
  std::vector<double> unused;
  if (deriv) {
    nz_tables(c, c->cos_p, c->nz_z[s], c->nz_n[s], tab[Q_PLUS], unused, chip);
    nz_tables(c, c->cos_m, c->nz_z[s], c->nz_n[s], tab[Q_MINUS], unused, chim);
    c->chi_s_p[s] = chip;
    c->chi_s_m[s] = chim;
    c->mean_p[s] = nz_mean_term(c, c->cos_p, cfg.omega_m + c->adj_h, tab[Q_PLUS]);
    c->mean_m[s] = nz_mean_term(c, c->cos_m, cfg.omega_m - c->adj_h, tab[Q_MINUS]);
  } else {
    tab[Q_PLUS].assign(kChiTab, 0.0);
    tab[Q_MINUS].assign(kChiTab, 0.0);
  }
  const size_t per = (size_t)cfg.n_zs * kChiTab;
  for (int kind = 0; kind < 4; ++kind) {
    const size_t at = (size_t)kind * per + (size_t)s * kChiTab;
    cudaError_t e = cudaMemcpyAsync(c->ws + c->L.qtab + at * 8, tab[kind].data(), kChiTab * 8,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e) return e;
    std::vector<float> f(tab[kind].begin(), tab[kind].end());
    if ((e = cudaMemcpyAsync(c->ws + c->L.qtab_f + at * 4, f.data(), kChiTab * 4, cudaMemcpyHostToDevice,
                             c->stream)))
      return e;
    if ((e = cudaStreamSynchronize(c->stream))) return e;  // the host vectors go out of scope
  }
  c->nz_mask |= 1u << s;
  return cudaSuccess;
}

// FP32 mirror of a chi table, uploaded beside the FP64 one
cudaError_t upload_ftab(pm_ctx* c, int id, const std::vector<double>& v) {
  std::vector<float> f(v.begin(), v.end());
  cudaError_t e = cudaMemcpyAsync(c->ws + c->L.ftab + id * al(kChiTab * 4), f.data(), f.size() * 4,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e) return e;
  return cudaStreamSynchronize(c->stream);  // f goes out of scope
}

// Omega_m +/- h coefficient sets for the finite-difference derivative
void build_adjoint_tables(pm_ctx* c) {
  const pm_config& cfg = c->cfg;
  c->adj_h = 1e-3;
  const int n = cfg.nsteps;
  for (int sgn = 0; sgn < 2; ++sgn) {
    const double om = cfg.omega_m + (sgn == 0 ? c->adj_h : -c->adj_h);
    Cosmo& co = sgn == 0 ? c->cos_p : c->cos_m;
    co.init(om, cfg.sigma8, cfg.h, cfg.n_s, cfg.omega_b, cfg.t_cmb);
    std::vector<double>& kk = sgn == 0 ? c->kick_p : c->kick_m;
    std::vector<double>& dd = sgn == 0 ? c->drift_p : c->drift_m;
    std::vector<double>& cs = sgn == 0 ? c->chi_s_p : c->chi_s_m;
    double* mt = sgn == 0 ? c->mean_p : c->mean_m;
    kk.resize(n);
    dd.resize(n);
    for (int i = 0; i < n; ++i) {
      const double aprev = i == 0 ? c->a[0] : c->ah[i - 1];
      kk[i] = (co.gp(c->ah[i]) - co.gp(aprev)) / co.gf(c->a[i]);
      dd[i] = (co.D1(c->a[i + 1]) - co.D1(c->a[i])) / co.gp(c->ah[i]);
    }
    cs.resize(cfg.n_zs);
    for (int s = 0; s < PM_MAX_ZS; ++s) mt[s] = 0.0;
    std::vector<double> ag(8001);
    for (int s = 0; s < cfg.n_zs; ++s) {
      cs[s] = co.chi_a(1.0 / (1.0 + cfg.zs[s]));
      const int m = 8000;
      const double hh = cs[s] / m;
      co.a_of_chi_grid(hh, m + 1, ag.data());
      double acc = 0;
      for (int q = 0; q <= m; ++q) {
        const double x = q * hh;
        acc += (q == 0 || q == m ? 1.0 : (q & 1 ? 4.0 : 2.0)) * x * (cs[s] - x) / (cs[s] * ag[q]);
      }
      mt[s] = 1.5 * om / (kCoverH0 * kCoverH0) * acc * hh / 3.0;
    }
  }
}

cudaError_t upload_adjoint_tables(pm_ctx* c) {
  const pm_config& cfg = c->cfg;
  std::vector<double> dd1(kChiTab), dinva(kChiTab), d1p(kChiTab), d1m(kChiTab), ivp(kChiTab), ivm(kChiTab);
  std::vector<double> ag(kChiTab), agp(kChiTab), agm(kChiTab);
  c->cosmo.a_of_chi_grid(c->chi_tab_h, kChiTab, ag.data());
  c->cos_p.a_of_chi_grid(c->chi_tab_h, kChiTab, agp.data());
  c->cos_m.a_of_chi_grid(c->chi_tab_h, kChiTab, agm.data());
  for (int k = 0; k < kChiTab; ++k) {
    const double a = ag[k];
    dd1[k] = -c->cosmo.gp(a) / (a * kCoverH0);  // dD1(a(chi))/dchi
    dinva[k] = c->cosmo.E(a) / kCoverH0;        // d(1/a)/dchi
    const double ap = agp[k], am = agm[k];
    d1p[k] = c->cos_p.D1(ap);
    d1m[k] = c->cos_m.D1(am);
    ivp[k] = 1.0 / ap;
    ivm[k] = 1.0 / am;
  }
  const int nh = cfg.nc / 2;
  std::vector<double> sp(3 * nh * nh + 1), sm(3 * nh * nh + 1);
  const double kf = 2.0 * M_PI / cfg.box, vol = cfg.box * cfg.box * cfg.box;
  const double ncube = (double)cfg.nc * cfg.nc * cfg.nc;
  sp[0] = sm[0] = 0.0;
  for (size_t n2 = 1; n2 < sp.size(); ++n2) {
    const double k = kf * std::sqrt((double)n2);
    sp[n2] = std::sqrt(c->cos_p.pk(k) * ncube / vol);
    sm[n2] = std::sqrt(c->cos_m.pk(k) * ncube / vol);
  }
  const std::pair<size_t, std::vector<double>*> up[] = {{c->L.tab_dd1, &dd1}, {c->L.tab_dinva, &dinva},
                                                        {c->L.tab_d1p, &d1p},  {c->L.tab_d1m, &d1m},
                                                        {c->L.tab_invap, &ivp}, {c->L.tab_invam, &ivm},
                                                        {c->L.sqrtp_p, &sp},   {c->L.sqrtp_m, &sm}};
  for (const auto& u : up) {
    cudaError_t e = cudaMemcpyAsync(c->ws + u.first, u.second->data(), u.second->size() * 8, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e) return e;
  }
  const std::pair<int, std::vector<double>*> fu[] = {{T_DD1, &dd1}, {T_DINVA, &dinva}, {T_D1P, &d1p},
                                                     {T_D1M, &d1m}, {T_INVAP, &ivp},   {T_INVAM, &ivm}};
  for (const auto& u : fu)
    if (cudaError_t e = upload_ftab(c, u.first, *u.second)) return e;
  return cudaStreamSynchronize(c->stream);
}

cudaError_t upload_tables(pm_ctx* c) {
  const pm_config& cfg = c->cfg;
  std::vector<double> d1t(kChiTab), inva(kChiTab), ag(kChiTab);
  c->cosmo.a_of_chi_grid(c->chi_tab_h, kChiTab, ag.data());
  for (int k = 0; k < kChiTab; ++k) {
    const double a = ag[k];
    d1t[k] = c->cosmo.D1(a);
    inva[k] = 1.0 / a;
  }
  const int nh = cfg.nc / 2;
  std::vector<double> sq(3 * nh * nh + 1);
  const double kf = 2.0 * M_PI / cfg.box, vol = cfg.box * cfg.box * cfg.box;
  const double ncube = (double)cfg.nc * cfg.nc * cfg.nc;
  sq[0] = 0.0;
  for (size_t n2 = 1; n2 < sq.size(); ++n2) sq[n2] = std::sqrt(c->cosmo.pk(kf * std::sqrt((double)n2)) * ncube / vol);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.tab_d1, d1t.data(), kChiTab * 8, cudaMemcpyHostToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.tab_inva, inva.data(), kChiTab * 8, cudaMemcpyHostToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.sqrtp, sq.data(), sq.size() * 8, cudaMemcpyHostToDevice, c->stream))) return e;
  if ((e = cudaMemsetAsync(c->ws + c->L.flags, 0, 256, c->stream))) return e;
  if ((e = upload_ftab(c, T_D1, d1t))) return e;
  if ((e = upload_ftab(c, T_INVA, inva))) return e;
  return cudaStreamSynchronize(c->stream);  // host vectors go out of scope
}

// ---------------------------------------------------------- force passes
// Paint is done by the caller into rho; this computes the force meshes (and
// the PGD meshes when alpha_pgd is given) from rho.
template <typename R>
cudaError_t force_from_rho(pm_ctx* c, bool with_pgd, double alpha_pgd, size_t s_off = 0, size_t f_off = 0) {
  const pm_config& cfg = c->cfg;
  SpecParams sp = {};
  sp.err = timeout_ptr(c);
  sp.op = with_pgd ? OP_FORCE_PGD : OP_FORCE;
  sp.kf = 2.0 * M_PI / cfg.box;
  const double m3 = (double)c->M * c->M * c->M;
  sp.scale = 1.5 * cfg.omega_m * (c->M / cfg.box) / m3;
  sp.pgd_scale = alpha_pgd * (c->M / cfg.box) / m3;
  sp.kl = cfg.pgd_params[2];
  sp.ks = cfg.pgd_params[3];
  sp.nexp = cfg.pgd_params[4];
  const int nout = with_pgd ? 6 : 3;
  void* ub[6];
  R* outs[6];
  for (int o = 0; o < nout; ++o) ub[o] = c->ws + c->L.ubuf + o * al(cmesh_bytes(c));
  // force (and PGD) meshes: the context's, or adjoint segment slots (three meshes of
  // mesh_elems each: the mesh bytes of every supported size are a multiple of 256)
  R* F = rp<R>(c, f_off ? f_off : c->L.fmesh);
  for (int o = 0; o < 3; ++o) outs[o] = F + o * c->mesh_elems;
  if (with_pgd) {
    R* S = rp<R>(c, s_off ? s_off : c->L.smesh);
    for (int o = 0; o < 3; ++o) outs[3 + o] = S + o * c->mesh_elems;
  }
  return spectral_apply<R>(rp<R>(c, c->L.rho), c->ws + c->L.cbuf, ub, outs, nout, c->M, c->P, sp, c->stream,
                           &c->prof);
}

bool shell_active(pm_ctx* c, int i) {
  double mx = 0;
  for (double v : c->chi_s) mx = std::max(mx, v);
  return c->chi_a[i + 1] < mx;
}

double pgd_alpha(pm_ctx* c, int i) { return c->cfg.pgd_params[0] * std::pow(c->a[i + 1], c->cfg.pgd_params[1]); }

template <typename R>
pm_status do_ic(pm_ctx* c, const double* d_noise) {
  const pm_config& cfg = c->cfg;
  cudaStream_t s = c->stream;
  const long long g = (long long)c->nc * c->nc * c->nc;
  R* noise = rp<R>(c, c->L.ic_real);
  cudaError_t e = launch_convert_in<R>(d_noise, noise, g, s, &c->prof);
  if (e) return PM_ERR_CUDA;
  const int nout = cfg.lpt_order == 2 ? 9 : 3;
  void* ub[9];
  R* outs[13];
  for (int o = 0; o < 9; ++o) ub[o] = c->ws + c->L.ic_u + o * al(cgrid_bytes(c));
  for (int o = 0; o < 13; ++o) outs[o] = rp<R>(c, c->L.ic_out + o * al(g * c->rsz));
  SpecParams sp = {};
  sp.err = timeout_ptr(c);
  sp.op = cfg.lpt_order == 2 ? OP_LPT2_DERIV : OP_LPT1;
  sp.kf = 2.0 * M_PI / cfg.box;
  sp.scale = 1.0 / (double)g;
  sp.sqrtp = reinterpret_cast<const double*>(c->ws + c->L.sqrtp);
  if ((e = spectral_apply<R>(noise, c->ws + c->L.ic_cbuf, ub, outs, nout, c->nc, c->Pc, sp, s, &c->prof, KK_IC)))
    return PM_ERR_CUDA;
  R* const* psi2 = nullptr;
  if (cfg.lpt_order == 2) {
    if ((e = launch_lpt2_source<R>(c, outs + 3, outs[9], g))) return PM_ERR_CUDA;
    SpecParams sp2 = sp;
    sp2.op = OP_GRAD_NEG;
    if ((e = spectral_apply<R>(outs[9], c->ws + c->L.ic_cbuf, ub, outs + 10, 3, c->nc, c->Pc, sp2, s, &c->prof,
                               KK_IC)))
      return PM_ERR_CUDA;
    psi2 = outs + 10;
  }
  const double a0 = c->a[0];
  const Cosmo& co = c->cosmo;
  if (c->tan_noise) {
    // tangent initial conditions along the noise direction (pm_jvp): the same
    // spectral operators on the direction, the 2LPT source linearised about
    // the base second derivatives outs[3..8]
    auto tf = [&](int q) { return rp<R>(c, c->L.tan_ic + (size_t)q * al(g * c->rsz)); };
    if ((e = launch_convert_in<R>(c->tan_noise, tf(0), g, s, &c->prof))) return PM_ERR_CUDA;
    R* touts[13];
    for (int o = 0; o < 13; ++o) touts[o] = tf(1 + o);
    if ((e = spectral_apply<R>(tf(0), c->ws + c->L.ic_cbuf, ub, touts, nout, c->nc, c->Pc, sp, s, &c->prof,
                               KK_JVP)))
      return PM_ERR_CUDA;
    if (cfg.lpt_order == 2) {
      if ((e = launch_lpt2_source_tan<R>(c, outs + 3, touts + 3, touts[9], g))) return PM_ERR_CUDA;
      SpecParams sp2 = sp;
      sp2.op = OP_GRAD_NEG;
      if ((e = spectral_apply<R>(touts[9], c->ws + c->L.ic_cbuf, ub, touts + 10, 3, c->nc, c->Pc, sp2, s,
                                 &c->prof, KK_JVP)))
        return PM_ERR_CUDA;
    }
    if ((e = launch_tan_ic<R>(c, touts, psi2 ? touts + 10 : nullptr, co.D1(a0), psi2 ? co.D2(a0) : 0.0, co.gp(a0),
                              psi2 ? co.gp2(a0) : 0.0)))
      return PM_ERR_CUDA;
  }
  if ((e = launch_ic_particles<R>(c, outs, psi2, co.D1(a0), psi2 ? co.D2(a0) : 0.0, co.gp(a0),
                                  psi2 ? co.gp2(a0) : 0.0)))
    return PM_ERR_CUDA;
  launch_iota(c);  // lattice order
  R* rho = rp<R>(c, c->L.rho);
  if ((e = cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, s))) return PM_ERR_CUDA;
  if ((e = launch_paint<R>(c, rho))) return PM_ERR_CUDA;
  // resident adjoint: F(x_0) goes straight into segment slot 0
  const size_t f_off = adj_resident(c->cfg) ? fseg_off(c, 0) : 0;
  if ((e = force_from_rho<R>(c, false, 0.0, 0, f_off))) return PM_ERR_CUDA;
  c->f_at = f_off;
  c->s_at = 0;
  return PM_OK;
}

template <typename R>
pm_status do_step(pm_ctx* c, int i) {
  R* rho = rp<R>(c, c->L.rho);
  cudaError_t e;
  if ((e = cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, c->stream))) return PM_ERR_CUDA;
  if ((e = launch_kdk_paint<R>(c, rho, c->kick[i], c->drift[i]))) return PM_ERR_CUDA;
  const bool pgd = c->cfg.pgd && shell_active(c, i);
  // resident adjoint: F(x_{i+1}) and S(x_{i+1}) land in the step's segment slots
  const bool res = adj_resident(c->cfg);
  const size_t f_off = res && i + 1 < c->cfg.nsteps ? fseg_off(c, i + 1) : 0;
  const size_t s_off = res && pgd ? sseg_off(c, i) : 0;
  if ((e = force_from_rho<R>(c, pgd, pgd ? pgd_alpha(c, i) : 0.0, s_off, f_off))) return PM_ERR_CUDA;
  c->f_at = f_off;
  c->s_at = s_off;
  c->pgd_valid = pgd;
  return PM_OK;
}

// every replica box that may hold a particle of shell (lo, hi] whose projected
// position can land on the map (FOV widened by one pixel and a margin that
// bounds the sub-evolution and PGD displacements)
std::vector<Replica> shell_replicas(pm_ctx* c, double lo, double hi) {
  const pm_config& cfg = c->cfg;
  const double L = cfg.box;
  const double fov = cfg.map_fov_deg * M_PI / 180.0;
  const double half = 0.5 * fov + fov / cfg.map_npix;
  const double t = std::tan(half);
  const double margin = std::max(0.1 * L, 10.0);
  const double cosc = 1.0 / std::sqrt(1.0 + 2.0 * t * t);
  const double z0 = std::max(0.0, lo * cosc - margin), z1 = hi + margin;
  const double w = hi * t + margin;
  std::vector<Replica> out;
  for (int nz = (int)std::floor(z0 / L); nz <= (int)std::floor(z1 / L); ++nz)
    for (int ny = (int)std::floor(-w / L); ny <= (int)std::floor(w / L); ++ny)
      for (int nx = (int)std::floor(-w / L); nx <= (int)std::floor(w / L); ++nx) {
        const int n3[3] = {nx, ny, nz};
        double dmin2 = 0, dmax2 = 0;
        for (int d = 0; d < 3; ++d) {
          const double a = n3[d] * L, b = a + L;
          const double nearv = a > 0 ? a : (b < 0 ? b : 0.0);
          const double farv = std::fabs(a) > std::fabs(b) ? a : b;
          dmin2 += nearv * nearv;
          dmax2 += farv * farv;
        }
        if (dmin2 > hi * hi || dmax2 < lo * lo) continue;
        Replica r;
        r.n[0] = (int16_t)nx; r.n[1] = (int16_t)ny; r.n[2] = (int16_t)nz;
        if (cfg.rotate) {
          // SplitMix64 output of seed ^ (20-bit fields nx, ny, nz)
          uint64_t key = ((uint64_t)(nx & 0xFFFFF) << 40) | ((uint64_t)(ny & 0xFFFFF) << 20) |
                         (uint64_t)(nz & 0xFFFFF);
          uint64_t z = (cfg.rotation_seed ^ key) + 0x9E3779B97F4A7C15ULL;
          z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
          z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
          z ^= z >> 31;
          static const uint8_t perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
          const int pi = (int)(z % 6);
          for (int d = 0; d < 3; ++d) {
            r.perm[d] = perms[pi][d];
            r.shift[d] = (int16_t)(((z >> (16 + 16 * d)) & 0xFFFF) % (uint64_t)cfg.nmesh);
          }
          r.flip = (uint8_t)((z >> 8) & 7);
        } else {
          for (int d = 0; d < 3; ++d) { r.perm[d] = (uint8_t)d; r.shift[d] = 0; }
          r.flip = 0;
        }
        out.push_back(r);
      }
  return out;
}

template <typename R>
pm_status do_lens(pm_ctx* c, int i) {
  LensShell sh;
  const double lo = c->chi_a[i + 1], hi = c->chi_a[i];
  sh.chi_lo2 = lo * lo;
  sh.chi_hi2 = hi * hi;
  sh.d1_next = c->cosmo.D1(c->a[i + 1]);
  sh.gp_half = c->cosmo.gp(c->ah[i]);
  const std::vector<Replica> reps = shell_replicas(c, lo, hi);
  for (size_t b = 0; b < reps.size(); b += kMaxReplicas) {
    sh.nrep = (int)std::min<size_t>(kMaxReplicas, reps.size() - b);
    for (int q = 0; q < sh.nrep; ++q) sh.rep[q] = reps[b + q];
    if (launch_lens<R>(c, sh, c->cfg.pgd && c->pgd_valid)) return PM_ERR_CUDA;
  }
  return PM_OK;
}

pm_status read_flags(pm_ctx* c);

// one shot-noise run (Sec. 4): uniformly random particles at rest, sorted for
// the projection's replica culling, projected through every shell without PGD,
// the mean-density terms subtracted
template <typename R>
pm_status do_shot_noise(pm_ctx* c, uint64_t seed, double* out) {
  if (cudaMemsetAsync(c->ws + c->L.maps, 0, (size_t)c->cfg.n_zs * c->cfg.map_npix * c->cfg.map_npix * 8, c->stream))
    return PM_ERR_CUDA;
  if (launch_random_particles<R>(c, seed)) return PM_ERR_CUDA;
  launch_iota(c);
  if (sort_particles<R>(c)) return PM_ERR_CUDA;
  c->pgd_valid = 0;
  for (int i = 0; i < c->cfg.nsteps; ++i) {
    if (!shell_active(c, i)) continue;
    const pm_status st = do_lens<R>(c, i);
    if (st) return st;
  }
  if (launch_kappa_finalize(c, out)) return PM_ERR_CUDA;
  return read_flags(c);
}

template <typename R>
__global__ void k_unpad_complex(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* in,
                                double* out, int n, int P) {
  const long long h = n / 2 + 1;
  const long long tot = (long long)n * n * h;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < tot; j += (long long)gridDim.x * blockDim.x) {
    const long long row = j / h, k = j - row * h;
    const auto v = in[row * P + k];
    out[2 * j] = v.x;
    out[2 * j + 1] = v.y;
  }
}

pm_status read_flags(pm_ctx* c);

// ---------------------------------------------------------------- adjoint
// copy the working particle state to / from a packed state block
cudaError_t save_state(pm_ctx* c, size_t dst) {
  const size_t np = c->np, r3 = 3 * np * c->rsz;
  char* d = c->ws + dst;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d, c->ws + c->L.cell, np * 4, cudaMemcpyDeviceToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(d + al(np * 4), c->ws + c->L.frac, r3, cudaMemcpyDeviceToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(d + al(np * 4) + al(r3), c->ws + c->L.mom, r3, cudaMemcpyDeviceToDevice, c->stream)))
    return e;
  return cudaMemcpyAsync(d + al(np * 4) + 2 * al(r3), c->ws + c->L.pid, np * 4, cudaMemcpyDeviceToDevice, c->stream);
}

cudaError_t load_state(pm_ctx* c, size_t src) {
  const size_t np = c->np, r3 = 3 * np * c->rsz;
  const char* s = c->ws + src;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.cell, s, np * 4, cudaMemcpyDeviceToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.frac, s + al(np * 4), r3, cudaMemcpyDeviceToDevice, c->stream))) return e;
  if ((e = cudaMemcpyAsync(c->ws + c->L.mom, s + al(np * 4) + al(r3), r3, cudaMemcpyDeviceToDevice, c->stream)))
    return e;
  return cudaMemcpyAsync(c->ws + c->L.pid, s + al(np * 4) + 2 * al(r3), np * 4, cudaMemcpyDeviceToDevice, c->stream);
}

const uint32_t* state_pid(pm_ctx* c, size_t off) {
  const size_t np = c->np, r3 = 3 * np * c->rsz;
  return reinterpret_cast<const uint32_t*>(c->ws + off + al(np * 4) + 2 * al(r3));
}

template <typename R>
AdjState<R> state_view(pm_ctx* c, size_t off) {
  const size_t np = c->np;
  const char* b = c->ws + off;
  AdjState<R> s;
  s.cell = reinterpret_cast<const uint32_t*>(b);
  const R* f = reinterpret_cast<const R*>(b + al(np * 4));
  const R* p = reinterpret_cast<const R*>(b + al(np * 4) + al(3 * np * c->rsz));
  s.fx = f; s.fy = f + np; s.fz = f + 2 * np;
  s.px = p; s.py = p + np; s.pz = p + 2 * np;
  return s;
}

size_t seg_off(pm_ctx* c, int j) { return c->L.adj_seg + (size_t)j * c->L.state_bytes; }
size_t fseg_off(pm_ctx* c, int j) { return c->L.adj_fseg + (size_t)j * 3 * al(c->mesh_elems * c->rsz); }
size_t sseg_off(pm_ctx* c, int j) { return c->L.adj_sseg + (size_t)j * 3 * al(c->mesh_elems * c->rsz); }

size_t ckpt_off(pm_ctx* c, int j) { return c->L.adj_ckpt + (size_t)j * c->L.state_bytes; }

SpecParams force_params(pm_ctx* c, bool pgd, double alpha) {
  SpecParams sp = {};
  sp.err = timeout_ptr(c);
  const double m3 = (double)c->M * c->M * c->M;
  sp.op = pgd ? OP_FORCE_PGD : OP_FORCE;
  sp.kf = 2.0 * M_PI / c->cfg.box;
  sp.scale = 1.5 * c->cfg.omega_m * (c->M / c->cfg.box) / m3;
  sp.pgd_scale = alpha * (c->M / c->cfg.box) / m3;
  sp.kl = c->cfg.pgd_params[2];
  sp.ks = c->cfg.pgd_params[3];
  sp.nexp = c->cfg.pgd_params[4];
  return sp;
}

// transpose of the mesh force (or PGD) at the state `st`: lam_x += F^T(v)
template <typename R>
cudaError_t mesh_vjp(pm_ctx* c, const AdjState<R>& st, const R* v, bool pgd_part, double alpha, R* const* meshes,
                     const R* lp_for_dot, double* dot) {
  cudaStream_t s = c->stream;
  R* pm[3];
  for (int q = 0; q < 3; ++q) pm[q] = rp<R>(c, c->L.adj_paint + q * al(c->mesh_elems * c->rsz));
  cudaError_t e;
  void* ub[6];
  for (int o = 0; o < 6; ++o) ub[o] = c->ws + c->L.ubuf + o * al(cmesh_bytes(c));
  R* phi = rp<R>(c, c->L.rho);
  const SpecParams sp = force_params(c, pgd_part, alpha);
  if constexpr (std::is_same<R, float>::value) {
    // FP32: the three cotangent components in one float4-interleaved mesh
    if ((e = cudaMemsetAsync(pm[0], 0, 4 * c->mesh_elems * sizeof(float), s))) return e;
    adj_paint_weights4(st, v, pm[0], c->M, c->np, s, &c->prof);
    if ((e = spectral_forward_xy_il<R>(pm[0], 4, 3, ub, c->M, c->P, sp, s, &c->prof))) return e;
    if ((e = spectral_transpose_pre<R>(pm, 3, 3, pgd_part ? 3 : 0, ub, c->ws + c->L.cbuf, phi, c->M, c->P, sp, s,
                                       &c->prof)))
      return e;
  } else {
    if ((e = cudaMemsetAsync(pm[0], 0, 3 * al(c->mesh_elems * c->rsz), s))) return e;
    adj_paint_weights<R>(st, v, pm, c->M, c->np, s, &c->prof);
    if ((e = spectral_transpose<R>(pm, 3, pgd_part ? 3 : 0, ub, c->ws + c->L.cbuf, phi, c->M, c->P, sp, s, &c->prof)))
      return e;
  }
  const double mass = std::pow((double)c->M / c->nc, 3.0);
  adj_readout_grad<R>(st, meshes, v, phi, mass, rp<R>(c, c->L.adj_lx), lp_for_dot, dot, c->M, c->np, s, &c->prof);
  return cudaGetLastError();
}

// The PGD transpose of a lightcone step and the kick transpose of the next step act at
// the same positions: one pass for both.  The kick's cotangents vF (with the force meshes
// Fm) and the PGD's vS (with the PGD meshes Sm) are painted in turn onto the same scratch
// meshes (the first set is x,y-transformed before the second is painted), one
// fused z pass sums the six conjugate multipliers, one inverse gives the potential, and
// one readout pass differentiates all seven meshes.  lam_x += F^T(vF) + S^T(vS);
// dot += sum_j vF_j . F(x_j).
template <typename R>
cudaError_t mesh_vjp_pair(pm_ctx* c, const AdjState<R>& st, const R* vF, R* const* Fm, const R* vS, R* const* Sm,
                          double alpha, double* dot) {
  cudaStream_t s = c->stream;
  R* pm[3];
  for (int q = 0; q < 3; ++q) pm[q] = rp<R>(c, c->L.adj_paint + q * al(c->mesh_elems * c->rsz));
  void* ub[6];
  for (int o = 0; o < 6; ++o) ub[o] = c->ws + c->L.ubuf + o * al(cmesh_bytes(c));
  const SpecParams sp = force_params(c, true, alpha);
  cudaError_t e;
  R* phi = rp<R>(c, c->L.rho);
  if constexpr (std::is_same<R, float>::value) {
    // FP32: both sets painted in one pass, vF_x, vF_y, vF_z, vS_x interleaved per cell as
    // float4 in the cotangent scratch and vS_y, vS_z as float2 in the density and spectrum
    // scratch (free until the transposed z pass writes its spectrum there; 2 x 4 M^3 bytes
    // fit, the spectrum alone being larger than one real mesh)
    float* m2 = rp<float>(c, c->L.rho);
    if ((e = cudaMemsetAsync(pm[0], 0, 4 * c->mesh_elems * sizeof(float), s))) return e;
    if ((e = cudaMemsetAsync(m2, 0, 2 * c->mesh_elems * sizeof(float), s))) return e;
    adj_paint_weights6(st, vF, vS, pm[0], m2, c->M, c->np, s, &c->prof);
    if ((e = spectral_forward_xy_il<R>(pm[0], 4, 4, ub, c->M, c->P, sp, s, &c->prof))) return e;
    if ((e = spectral_forward_xy_il<R>(m2, 2, 2, ub + 4, c->M, c->P, sp, s, &c->prof))) return e;
    R* ins[6] = {};
    if ((e = spectral_transpose_pre<R>(ins, 6, 6, 0, ub, c->ws + c->L.cbuf, phi, c->M, c->P, sp, s, &c->prof)))
      return e;
  } else {
    if ((e = cudaMemsetAsync(pm[0], 0, 3 * al(c->mesh_elems * c->rsz), s))) return e;
    adj_paint_weights<R>(st, vF, pm, c->M, c->np, s, &c->prof);
    if ((e = spectral_forward_xy<R>(pm, 3, ub, c->M, c->P, sp, s, &c->prof))) return e;
    if ((e = cudaMemsetAsync(pm[0], 0, 3 * al(c->mesh_elems * c->rsz), s))) return e;
    adj_paint_weights<R>(st, vS, pm, c->M, c->np, s, &c->prof);
    R* ins[6] = {nullptr, nullptr, nullptr, pm[0], pm[1], pm[2]};
    if ((e = spectral_transpose_pre<R>(ins, 6, 3, 0, ub, c->ws + c->L.cbuf, phi, c->M, c->P, sp, s, &c->prof)))
      return e;
  }
  const double mass = std::pow((double)c->M / c->nc, 3.0);
  adj_readout_grad2<R>(st, Fm, vF, Sm, vS, phi, mass, rp<R>(c, c->L.adj_lx), vF, dot, c->M, c->np, s, &c->prof);
  return cudaGetLastError();
}

LensShell make_shell(pm_ctx* c, int i, const Cosmo& co) {
  LensShell sh;
  const double lo = c->chi_a[i + 1], hi = c->chi_a[i];
  sh.chi_lo2 = lo * lo;
  sh.chi_hi2 = hi * hi;
  sh.d1_next = co.D1(c->a[i + 1]);
  sh.gp_half = co.gp(c->ah[i]);
  sh.nrep = 0;
  return sh;
}

template <typename R>
pm_status do_vjp(pm_ctx* c, const double* lam, double* d_noise_out, double* h_params) {
  const pm_config& cfg = c->cfg;
  cudaStream_t s = c->stream;
  Prof* pf = &c->prof;
  const long long np = c->np, np3 = 3 * np;
  const int n = cfg.nsteps, k = cfg.ckpt_every;
  const long long npix2 = (long long)cfg.map_npix * cfg.map_npix;
  R* lx = rp<R>(c, c->L.adj_lx);
  R* lp = rp<R>(c, c->L.adj_lp);
  R* v = rp<R>(c, c->L.adj_v);
  R* vS = rp<R>(c, c->L.adj_vs);
  double* acc = reinterpret_cast<double*>(c->ws + c->L.adj_acc);
  // acc layout: [0,n) kick dots, [n,2n) drift dots, [2n,3n) lens(+h), [3n,4n) lens(-h),
  //             4n + s: sum of lam over source s, 4n+16..: IC terms
  double* acc_ic = acc + 4 * n + 16;
  cudaError_t e;
  if ((e = cudaMemsetAsync(lx, 0, np3 * c->rsz, s))) return PM_ERR_CUDA;
  if ((e = cudaMemsetAsync(lp, 0, np3 * c->rsz, s))) return PM_ERR_CUDA;
  if ((e = cudaMemsetAsync(acc, 0, (size_t)(4 * n + 64) * 8, s))) return PM_ERR_CUDA;
  for (int q = 0; q < cfg.n_zs; ++q) adj_dsum(lam + q * npix2, npix2, acc + 4 * n + q, s, pf);
  // the projection transposes read lam in the path precision (FP32: rounded once here
  // instead of converted at every read)
  const R* lam_r;
  if constexpr (std::is_same<R, float>::value) {
    float* l32 = rp<float>(c, c->L.adj_lam);
    if ((e = launch_convert_in<float>(lam, l32, cfg.n_zs * npix2, s, pf))) return PM_ERR_CUDA;
    lam_r = l32;
  } else {
    lam_r = lam;
  }
  R* F = rp<R>(c, c->L.fmesh);
  R* Fm[3] = {F, F + c->mesh_elems, F + 2 * c->mesh_elems};
  const double vp = std::pow(cfg.box / c->nc, 3.0);
  const double dth = cfg.map_fov_deg * M_PI / 180.0 / cfg.map_npix;
  const double wpref_p = 1.5 * (cfg.omega_m + c->adj_h) / (kCoverH0 * kCoverH0) * vp / (dth * dth);
  const double wpref_m = 1.5 * (cfg.omega_m - c->adj_h) / (kCoverH0 * kCoverH0) * vp / (dth * dth);
  const int nck = c->L.nck;
  const bool resident = adj_resident(cfg) && (int)c->sorted_after.size() == n;
  for (int seg = nck - 1; seg >= 0; --seg) {
    const int i0 = seg * k, i1 = std::min(n, i0 + k);
    if (seg < nck - 1) {
      // the adjoint state is in checkpoint seg+1's particle order; bring it to seg's
      const uint32_t* pid_next = state_pid(c, ckpt_off(c, seg + 1));
      const uint32_t* pid_here = state_pid(c, ckpt_off(c, seg));
      for (R* a : {lx, lp}) {
        if (launch_unpermute3<R>(c, a, pid_next, v)) return PM_ERR_CUDA;
        if (launch_permute3<R>(c, v, pid_here, a)) return PM_ERR_CUDA;
      }
    }
    // recompute the segment forward from its checkpoint, keeping every state
    // (resident mode: the forward already kept them)
    // The force meshes F(x_i) are written straight into their segment slots (the force
    // evaluation's output pointers), where the next kick reads them: no copies.
    if (!resident) {
    if ((e = load_state(c, ckpt_off(c, seg)))) return PM_ERR_CUDA;
    {
      R* rho = rp<R>(c, c->L.rho);
      if ((e = cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, s))) return PM_ERR_CUDA;
      if ((e = launch_paint<R>(c, rho))) return PM_ERR_CUDA;
      if ((e = force_from_rho<R>(c, false, 0.0, 0, fseg_off(c, 0)))) return PM_ERR_CUDA;
      c->f_at = fseg_off(c, 0);
    }
    if ((e = save_state(c, seg_off(c, 0)))) return PM_ERR_CUDA;
    for (int i = i0; i < i1; ++i) {
      R* rho = rp<R>(c, c->L.rho);
      if ((e = cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, s))) return PM_ERR_CUDA;
      if ((e = launch_kdk_paint<R>(c, rho, c->kick[i], c->drift[i]))) return PM_ERR_CUDA;  // reads F at f_at
      // lens steps with PGD: S(x_{i+1}) comes with the force, kept for the reverse sweep;
      // F(x_{i+1}) for kick i + 1 goes to slot i + 1 of the segment
      const bool pg_i = cfg.pgd && shell_active(c, i);
      const size_t f_off = i + 1 < i1 ? fseg_off(c, i - i0 + 1) : 0;
      if ((e = force_from_rho<R>(c, pg_i, pg_i ? pgd_alpha(c, i) : 0.0, pg_i ? sseg_off(c, i - i0) : 0, f_off)))
        return PM_ERR_CUDA;
      c->f_at = f_off;
      if ((e = save_state(c, seg_off(c, i - i0 + 1)))) return PM_ERR_CUDA;
    }
    }
    // reverse sweep through the segment.  The kick transpose of step i + 1 acts at x_{i+1},
    // where the PGD transpose of shell i acts too: when step i lies in this segment with an
    // active PGD shell, the kick's cotangent v waits in its buffer and both run as one pass
    // (mesh_vjp_pair) right after shell i's lens transpose, still before the drift transpose
    // of step i that reads lam_x(x_{i+1}).
    int pending = -1;  // step whose kick transpose waits in v
    for (int i = i1 - 1; i >= i0; --i) {
      const AdjState<R> st1 = state_view<R>(c, seg_off(c, i - i0 + 1));  // x_{i+1}, p_{i+1/2}
      const size_t mstride = al(c->mesh_elems * c->rsz) / c->rsz;
      if (shell_active(c, i)) {
        const bool pg = cfg.pgd != 0;
        // S(x_{i+1}) from the segment recompute
        R* Sseg = rp<R>(c, sseg_off(c, i - i0));
        const size_t sstride = al(c->mesh_elems * c->rsz) / c->rsz;
        R* Sm[3] = {Sseg, Sseg + sstride, Sseg + 2 * sstride};
        c->s_at = pg ? sseg_off(c, i - i0) : 0;
        LensShell sh = make_shell(c, i, c->cosmo);
        const std::vector<Replica> reps = shell_replicas(c, std::sqrt(sh.chi_lo2), std::sqrt(sh.chi_hi2));
        LensAdjArgs<R> A;
        A.st = st1;
        A.S0 = pg ? Sm[0] : nullptr;
        A.S1 = pg ? Sm[1] : nullptr;
        A.S2 = pg ? Sm[2] : nullptr;
        A.np = np;
        A.M = c->M;
        A.cell_len = cfg.box / c->M;
        A.chi_lo2 = sh.chi_lo2;
        A.chi_hi2 = sh.chi_hi2;
        const double fov = cfg.map_fov_deg * M_PI / 180.0;
        A.fov_half = 0.5 * fov;
        A.inv_dtheta = 1.0 / dth;
        A.tan_half = std::tan(0.5 * fov + dth);
        A.margin = std::max(0.1 * cfg.box, 10.0);
        A.npix = cfg.map_npix;
        A.nzs = cfg.n_zs;
        A.sub = cfg.sub_evolution;
        for (int q = 0; q < PM_MAX_ZS; ++q) A.chi_s[q] = q < cfg.n_zs ? c->chi_s[q] : 0.0;
        A.wpref = 1.5 * cfg.omega_m / (kCoverH0 * kCoverH0) * vp / (dth * dth);
        A.d1_next = sh.d1_next;
        A.inv_gp_half = 1.0 / sh.gp_half;
        A.tab_hinv = 1.0 / c->chi_tab_h;
        for (int q = 0; q < PM_MAX_ZS; ++q) A.chi_s_r[q] = (R)A.chi_s[q];
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
        A.lam = lam_r;
        A.lx = lx;
        A.lp = lp;
        A.vS = pg ? vS : nullptr;
        if (pg && (e = cudaMemsetAsync(vS, 0, np3 * c->rsz, s))) return PM_ERR_CUDA;
        // the working state holds x_{i+1} for the dot passes
        if ((e = load_state(c, seg_off(c, i - i0 + 1)))) return PM_ERR_CUDA;
        LensShell shp = make_shell(c, i, c->cos_p), shm = make_shell(c, i, c->cos_m);
        for (size_t b = 0; b < reps.size(); b += kMaxReplicas) {
          A.nrep = (int)std::min<size_t>(kMaxReplicas, reps.size() - b);
          for (int q = 0; q < A.nrep; ++q) A.rep[q] = reps[b + q];
          adj_lens<R>(A, s, pf);
          shp.nrep = shm.nrep = A.nrep;
          for (int q = 0; q < A.nrep; ++q) shp.rep[q] = shm.rep[q] = A.rep[q];
          const LensDotVar vp_ = {T_D1P, T_INVAP, Q_PLUS, c->chi_s_p.data(), wpref_p, shp.d1_next, shp.gp_half,
                                  acc + 2 * n + i};
          const LensDotVar vm_ = {T_D1M, T_INVAM, Q_MINUS, c->chi_s_m.data(), wpref_m, shm.d1_next, shm.gp_half,
                                  acc + 3 * n + i};
          if (launch_lens_dot2<R>(c, shp, pg, lam_r, vp_, vm_)) return PM_ERR_CUDA;
        }
        if (pg) {
          // PGD transpose at x_{i+1}, with the waiting kick transpose of step i + 1 if any
          if (pending == i + 1) {
            R* Fn = rp<R>(c, fseg_off(c, i + 1 - i0));  // F(x_{i+1})
            R* Fns[3] = {Fn, Fn + mstride, Fn + 2 * mstride};
            if ((e = mesh_vjp_pair<R>(c, st1, v, Fns, vS, Sm, pgd_alpha(c, i), acc + i + 1))) return PM_ERR_CUDA;
            pending = -1;
          } else if ((e = mesh_vjp<R>(c, st1, vS, true, pgd_alpha(c, i), Sm, nullptr, nullptr))) {
            return PM_ERR_CUDA;
          }
        }
      }
      if (pending == i + 1) {  // no PGD transpose at x_{i+1} after all: the kick's alone
        R* Fn = rp<R>(c, fseg_off(c, i + 1 - i0));
        R* Fns[3] = {Fn, Fn + mstride, Fn + 2 * mstride};
        if ((e = mesh_vjp<R>(c, st1, v, false, 0.0, Fns, v, acc + i + 1))) return PM_ERR_CUDA;
        pending = -1;
      }
      // drift x_{i+1} = x_i + drift_i p_{i+1/2}
      adj_dot<R>(lx, st1.px, np3, acc + n + i, s, pf);
      adj_axpy<R>(lp, lx, c->drift[i], np3, s, pf);
      if (resident && c->sorted_after[i]) {
        // the state was re-sorted after step i: bring the adjoint to x_i's particle order
        const uint32_t* pid1 = state_pid(c, seg_off(c, i + 1));
        const uint32_t* pid0 = state_pid(c, seg_off(c, i));
        for (R* a : {lx, lp}) {
          if (launch_unpermute3<R>(c, a, pid1, v)) return PM_ERR_CUDA;
          if (launch_permute3<R>(c, v, pid0, a)) return PM_ERR_CUDA;
        }
      }
      // kick p_{i+1/2} = p_{i-1/2} + kick_i F(x_i): cotangent v = kick_i lam_p; the kick dot is
      // accumulated as sum v . F (the host divides by kick_i)
      adj_scale<R>(v, lp, c->kick[i], np3, s, pf);
      if (i > i0 && shell_active(c, i - 1) && cfg.pgd) {
        pending = i;  // runs with shell i - 1's PGD transpose, at x_i
      } else {
        const AdjState<R> st0 = state_view<R>(c, seg_off(c, i - i0));
        R* Fi = rp<R>(c, fseg_off(c, i - i0));  // F(x_i), kept by the segment recompute
        R* Fs[3] = {Fi, Fi + mstride, Fi + 2 * mstride};
        if ((e = mesh_vjp<R>(c, st0, v, false, 0.0, Fs, v, acc + i))) return PM_ERR_CUDA;
      }
    }
    if (pending >= 0) return PM_ERR_STATE;  // every deferred transpose ran inside its segment
  }
  // ------------------------------------------------ initial conditions
  const long long g = (long long)c->nc * c->nc * c->nc;
  auto field = [&](int q) { return rp<R>(c, c->L.adj_ic + (size_t)q * al(g * c->rsz)); };
  // fields: 0-2 Psi1, 3-8 second derivatives, 9 source, 10-12 Psi2, 13-15 lamPsi1, 16-18 lamPsi2,
  //         19 lamSrc, 20-25 lamDeriv, 26 d/dnoise, 27 spare
  const bool two = cfg.lpt_order == 2;
  void* ub[9];
  for (int o = 0; o < 9; ++o) ub[o] = c->ws + c->L.ic_u + o * al(cgrid_bytes(c));
  auto lpt_forward = [&](const double* sqrtp) -> cudaError_t {
    SpecParams sp = {};
    sp.err = timeout_ptr(c);
    sp.op = two ? OP_LPT2_DERIV : OP_LPT1;
    sp.kf = 2.0 * M_PI / cfg.box;
    sp.scale = 1.0 / (double)g;
    sp.sqrtp = sqrtp;
    R* outs[9];
    for (int q = 0; q < 9; ++q) outs[q] = field(q);
    cudaError_t ee = spectral_apply<R>(rp<R>(c, c->L.adj_noise), c->ws + c->L.ic_cbuf, ub, outs, two ? 9 : 3, c->nc,
                                       c->Pc, sp, s, pf, KK_ADJ_FFT);
    if (ee || !two) return ee;
    R* d[6];
    for (int q = 0; q < 6; ++q) d[q] = field(3 + q);
    if ((ee = launch_lpt2_source<R>(c, d, field(9), g))) return ee;
    SpecParams sp2 = sp;
    sp2.op = OP_GRAD_NEG;
    R* o2[3] = {field(10), field(11), field(12)};
    return spectral_apply<R>(field(9), c->ws + c->L.ic_cbuf, ub, o2, 3, c->nc, c->Pc, sp2, s, pf, KK_ADJ_FFT);
  };
  const double cpl = c->M / cfg.box;
  const double a0 = c->a[0];
  const Cosmo& co = c->cosmo;
  // Omega_m through the initial state: central differences of the LPT displacements
  for (int sgn = 0; sgn < 2; ++sgn) {
    const Cosmo& cx = sgn == 0 ? c->cos_p : c->cos_m;
    if ((e = lpt_forward(reinterpret_cast<const double*>(c->ws + (sgn == 0 ? c->L.sqrtp_p : c->L.sqrtp_m)))))
      return PM_ERR_CUDA;
    R* p1[3] = {field(0), field(1), field(2)};
    R* p2[3] = {field(10), field(11), field(12)};
    adj_ic_dot<R>(lx, lp, p1, two ? p2 : nullptr, cx.D1(a0), two ? cx.D2(a0) : 0.0, cx.gp(a0),
                  two ? cx.gp2(a0) : 0.0, cpl, g, acc_ic + sgn, s, pf);
  }
  if ((e = lpt_forward(reinterpret_cast<const double*>(c->ws + c->L.sqrtp)))) return PM_ERR_CUDA;
  R* lpsi1[3] = {field(13), field(14), field(15)};
  R* lpsi2[3] = {field(16), field(17), field(18)};
  adj_combine2<R>(lx, lp, lpsi1, co.D1(a0), co.gp(a0), cpl, g, s, pf);
  for (int q = 0; q < 3; ++q) adj_dot<R>(lpsi1[q], field(q), g, acc_ic + 2, s, pf);
  SpecParams sp = {};
  sp.err = timeout_ptr(c);
  sp.kf = 2.0 * M_PI / cfg.box;
  sp.scale = 1.0 / (double)g;
  sp.sqrtp = reinterpret_cast<const double*>(c->ws + c->L.sqrtp);
  R* wbar = field(26);
  if (!two) {
    sp.op = OP_LPT1;
    if ((e = spectral_transpose<R>(lpsi1, 3, 0, ub, c->ws + c->L.ic_cbuf, wbar, c->nc, c->Pc, sp, s, pf)))
      return PM_ERR_CUDA;
  } else {
    adj_combine2<R>(lx, lp, lpsi2, co.D2(a0), co.gp2(a0), cpl, g, s, pf);
    for (int q = 0; q < 3; ++q) adj_dot<R>(lpsi2[q], field(10 + q), g, acc_ic + 3, s, pf);
    SpecParams sg = sp;
    sg.op = OP_GRAD_NEG;
    if ((e = spectral_transpose<R>(lpsi2, 3, 0, ub, c->ws + c->L.ic_cbuf, field(19), c->nc, c->Pc, sg, s, pf)))
      return PM_ERR_CUDA;
    R* d[6];
    R* ld[6];
    for (int q = 0; q < 6; ++q) { d[q] = field(3 + q); ld[q] = field(20 + q); }
    adj_lpt2_src<R>(field(19), d, ld, g, s, pf);
    R* ins[9] = {lpsi1[0], lpsi1[1], lpsi1[2], ld[0], ld[1], ld[2], ld[3], ld[4], ld[5]};
    sp.op = OP_LPT2_DERIV;
    if ((e = spectral_transpose<R>(ins, 9, 0, ub, c->ws + c->L.ic_cbuf, wbar, c->nc, c->Pc, sp, s, pf)))
      return PM_ERR_CUDA;
  }
  if (d_noise_out && (e = launch_convert_out<R>(wbar, d_noise_out, g, 1.0, s, pf))) return PM_ERR_CUDA;
  // ------------------------------------------------ host combination
  std::vector<double> h(4 * n + 64);
  if (cudaMemcpyAsync(h.data(), acc, h.size() * 8, cudaMemcpyDeviceToHost, s)) return PM_ERR_CUDA;
  if (cudaStreamSynchronize(s)) return PM_ERR_CUDA;
  const double hh = c->adj_h, om = cfg.omega_m;
  double dom = 0.0;
  for (int i = 0; i < n; ++i) {
    const double dK = (c->kick_p[i] * (om + hh) - c->kick_m[i] * (om - hh)) / (2 * hh);  // d(kick Om)/dOm
    dom += dK / om * h[i] / c->kick[i];  // h[i] = kick_i sum lam_p . F(x_i)
    dom += (c->drift_p[i] - c->drift_m[i]) / (2 * hh) * h[n + i];
    dom += (h[2 * n + i] - h[3 * n + i]) / (2 * hh);
  }
  for (int q = 0; q < cfg.n_zs; ++q) dom -= h[4 * n + q] * (c->mean_p[q] - c->mean_m[q]) / (2 * hh);
  const double* hic = h.data() + 4 * n + 16;
  dom += (hic[0] - hic[1]) / (2 * hh);
  const double ds8 = (hic[2] + (two ? 2.0 * hic[3] : 0.0)) / cfg.sigma8;
  if (h_params) {
    h_params[0] = dom;
    h_params[1] = ds8;
  }
  return read_flags(c);
}

pm_status read_flags(pm_ctx* c) {
  int h[2] = {0, 0};  // non-finite word, timeout word
  if (cudaMemcpyAsync(h, c->ws + c->L.flags, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) return PM_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream)) return PM_ERR_CUDA;
  return h[1] ? PM_ERR_TIMEOUT : (h[0] ? PM_ERR_NONFINITE : PM_OK);
}

#define PM_DISPATCH(c, FN, ...) ((c)->prec == PM_FP64 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

template <typename R>
pm_status do_set_particles(pm_ctx* c, const double* x, const double* p, int ns) {
  if (launch_set_particles<R>(c, x, p)) return PM_ERR_CUDA;
  launch_iota(c);
  R* rho = rp<R>(c, c->L.rho);
  if (cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, c->stream)) return PM_ERR_CUDA;
  if (launch_paint<R>(c, rho)) return PM_ERR_CUDA;
  const bool pgd = ns > 0 && c->cfg.pgd && shell_active(c, ns - 1);
  if (force_from_rho<R>(c, pgd, pgd ? pgd_alpha(c, ns - 1) : 0.0)) return PM_ERR_CUDA;
  c->f_at = c->s_at = 0;
  c->pgd_valid = pgd;
  return PM_OK;
}

template <typename R>
pm_status do_readout(pm_ctx* c, size_t off, double* out) {
  R* m = rp<R>(c, off);
  R* ms[3] = {m, m + c->mesh_elems, m + 2 * c->mesh_elems};
  return cuda_status(launch_readout<R>(c, ms, c->cfg.box / c->M, out));
}

template <typename R>
pm_status do_fft(pm_ctx* c, const double* in, double* out) {
  R* rho = rp<R>(c, c->L.rho);
  if (launch_convert_in<R>(in, rho, c->mesh_elems, c->stream, &c->prof)) return PM_ERR_CUDA;
  if (fft3d_r2c<R>(rho, c->ws + c->L.cbuf, c->M, c->P, c->stream, &c->prof, timeout_ptr(c))) return PM_ERR_CUDA;
  using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
  ProfScope ps(&c->prof, KK_MISC, c->stream);
  k_unpad_complex<R><<<1024, 256, 0, c->stream>>>(reinterpret_cast<const C*>(c->ws + c->L.cbuf), out, c->M, c->P);
  return cuda_status(cudaGetLastError());
}

template <typename R>
pm_status do_density(pm_ctx* c, double* out) {
  R* rho = rp<R>(c, c->L.rho);
  if (cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, c->stream)) return PM_ERR_CUDA;
  if (launch_paint<R>(c, rho)) return PM_ERR_CUDA;
  return cuda_status(launch_convert_out<R>(rho, out, c->mesh_elems, 1.0, c->stream, &c->prof));
}

// d rho at the current positions from dx, then the force (and PGD) operator on it:
// dF (dS) meshes into the tangent slots
template <typename R>
cudaError_t tan_force(pm_ctx* c, bool pgd, double alpha) {
  R* rho = rp<R>(c, c->L.rho);
  cudaError_t e;
  if ((e = cudaMemsetAsync(rho, 0, c->mesh_elems * c->rsz, c->stream))) return e;
  if ((e = launch_tan_paint<R>(c, rho))) return e;
  return force_from_rho<R>(c, pgd, alpha, pgd ? c->L.tan_s : 0, c->L.tan_f);
}

template <typename R>
pm_status do_tan_lens(pm_ctx* c, int i) {
  LensShell sh = make_shell(c, i, c->cosmo);
  const std::vector<Replica> reps = shell_replicas(c, std::sqrt(sh.chi_lo2), std::sqrt(sh.chi_hi2));
  for (size_t b = 0; b < reps.size(); b += kMaxReplicas) {
    sh.nrep = (int)std::min<size_t>(kMaxReplicas, reps.size() - b);
    for (int q = 0; q < sh.nrep; ++q) sh.rep[q] = reps[b + q];
    if (launch_tan_lens<R>(c, sh, c->cfg.pgd && c->pgd_valid)) return PM_ERR_CUDA;
  }
  return PM_OK;
}

// forward run with the tangent state alongside (see pm_jvp)
template <typename R>
pm_status do_jvp(pm_ctx* c, const double* noise, const double* dnoise, double* kappa, double* dkappa) {
  const pm_config& cfg = c->cfg;
  const size_t map_bytes = (size_t)cfg.n_zs * cfg.map_npix * cfg.map_npix * 8;
  if (cudaMemsetAsync(c->ws + c->L.tan_maps, 0, map_bytes, c->stream)) return PM_ERR_CUDA;
  c->tan_noise = dnoise;
  pm_status st = pm_ic(c, noise);  // primal IC and the tangent dx0, dp0
  c->tan_noise = nullptr;
  if (st) return st;
  c->tan_on = 1;
  if (tan_force<R>(c, false, 0.0)) return PM_ERR_CUDA;  // dF(x_0)
  for (int i = 0; i < cfg.nsteps; ++i) {
    if (launch_tan_kd<R>(c, c->kick[i], c->drift[i])) return PM_ERR_CUDA;  // at x_i, before the primal moves
    if ((st = pm_step(c, i))) return st;                                   // x_{i+1}; re-sorts the tangent too
    const bool pgd = cfg.pgd && shell_active(c, i);
    if (tan_force<R>(c, pgd, pgd ? pgd_alpha(c, i) : 0.0)) return PM_ERR_CUDA;  // dF(x_{i+1}), dS(x_{i+1})
    if ((st = lens_project(c, i))) return st;
    if (shell_active(c, i) && (st = do_tan_lens<R>(c, i))) return st;
  }
  if (cudaMemcpyAsync(dkappa, c->ws + c->L.tan_maps, map_bytes, cudaMemcpyDeviceToDevice, c->stream))
    return PM_ERR_CUDA;
  return kappa_maps(c, kappa);
}

}  // namespace

extern "C" {

pm_status pm_workspace_size(const pm_config* cfg, size_t* bytes) {
  pm_status st = check_config(cfg);
  if (st) return st;
  if (!bytes) return PM_ERR_ARG;
  Layout L;
  int P, Pc;
  plan_layout(*cfg, L, P, Pc);
  *bytes = L.total;
  return PM_OK;
}

pm_status pm_init(pm_ctx** out, const pm_config* cfg, void* d_workspace, size_t bytes, void* stream) {
  if (!out) return PM_ERR_ARG;
  *out = nullptr;
  pm_status st = check_config(cfg);
  if (st) return st;
  Layout L;
  int P, Pc;
  plan_layout(*cfg, L, P, Pc);
  if (!d_workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) return PM_ERR_WORKSPACE;
  pm_ctx* c = new (std::nothrow) pm_ctx();
  if (!c) return PM_ERR_ARG;
  c->cfg = *cfg;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->prec = cfg->precision;
  c->rsz = cfg->precision == PM_FP64 ? 8 : 4;
  c->nc = cfg->nc;
  c->M = cfg->nmesh;
  c->np = (long long)cfg->nc * cfg->nc * cfg->nc;
  c->P = P;
  c->Pc = Pc;
  c->mesh_elems = (long long)c->M * c->M * c->M;
  c->cmesh_elems = (long long)c->M * c->M * P;
  c->cgrid_elems = (long long)c->nc * c->nc * Pc;
  c->nout_step = cfg->pgd ? 6 : 3;
  c->ws = reinterpret_cast<char*>(d_workspace);
  c->ws_bytes = bytes;
  c->L = L;
  c->next_step = -1;
  c->last_stepped = -1;
  c->projected = -1;
  c->pgd_valid = 0;
  c->ic_done = 0;
  c->vjp_state_lost = 0;
  build_tables(c);
  if (upload_tables(c) != cudaSuccess) { delete c; return PM_ERR_CUDA; }
  if (cfg->ckpt_every > 0 || cfg->jvp) {
    build_adjoint_tables(c);
    if (upload_adjoint_tables(c) != cudaSuccess) { delete c; return PM_ERR_CUDA; }
  }
  *out = c;
  return PM_OK;
}

pm_status pm_ic(pm_ctx* c, const double* d_noise) {
  if (!c || !d_noise) return PM_ERR_ARG;
  if (cudaMemsetAsync(c->ws + c->L.maps, 0, (size_t)c->cfg.n_zs * c->cfg.map_npix * c->cfg.map_npix * 8, c->stream))
    return PM_ERR_CUDA;
  pm_status st = PM_DISPATCH(c, do_ic, c, d_noise);
  if (st) return st;
  if (c->cfg.ckpt_every > 0) {
    // keep the noise and the initial state for the adjoint
    const long long g = (long long)c->nc * c->nc * c->nc;
    cudaError_t e = c->prec == PM_FP64
                        ? launch_convert_in<double>(d_noise, rp<double>(c, c->L.adj_noise), g, c->stream, &c->prof)
                        : launch_convert_in<float>(d_noise, rp<float>(c, c->L.adj_noise), g, c->stream, &c->prof);
    if (e || save_state(c, ckpt_off(c, 0))) return PM_ERR_CUDA;
    if (adj_resident(c->cfg) && save_state(c, seg_off(c, 0))) return PM_ERR_CUDA;
    c->sorted_after.assign(c->cfg.nsteps, 0);
  }
  c->ic_done = 1;
  c->next_step = 0;
  c->last_stepped = -1;
  c->projected = -1;
  c->pgd_valid = 0;
  c->vjp_state_lost = 0;
  return PM_OK;
}

pm_status pm_step(pm_ctx* c, int32_t i) {
  if (!c) return PM_ERR_ARG;
  if (i < 0 || i >= c->cfg.nsteps) return PM_ERR_ARG;
  if (!c->ic_done || i != c->next_step) return PM_ERR_STATE;
  pm_status st = PM_DISPATCH(c, do_step, c, i);
  if (st) return st;
  // restore spatial locality of the particle order (at checkpoint boundaries when the
  // adjoint is on, so that every checkpoint segment keeps one particle order)
  const int se = sort_every(c->cfg);
  const bool sorted = (i + 1) % se == 0 && i + 1 < c->cfg.nsteps;
  if (sorted) {
    cudaError_t e = c->prec == PM_FP64 ? sort_particles<double>(c) : sort_particles<float>(c);
    if (e) return PM_ERR_CUDA;
    if (c->tan_on) {
      // the sort swapped the state buffers: the old order's pid is now in L.pid2
      const uint32_t* old_pid = reinterpret_cast<const uint32_t*>(c->ws + c->L.pid2);
      const uint32_t* new_pid = reinterpret_cast<const uint32_t*>(c->ws + c->L.pid);
      e = c->prec == PM_FP64 ? tan_permute<double>(c, old_pid, new_pid) : tan_permute<float>(c, old_pid, new_pid);
      if (e) return PM_ERR_CUDA;
    }
  }
  if (adj_resident(c->cfg)) {
    // keep x_{i+1}, p_{i+1/2} in the order step i+1 uses
    if (save_state(c, seg_off(c, i + 1))) return PM_ERR_CUDA;
    if ((int)c->sorted_after.size() == c->cfg.nsteps) c->sorted_after[i] = sorted ? 1 : 0;
  }
  const int k = c->cfg.ckpt_every;
  if (k > 0 && (i + 1) % k == 0 && i + 1 < c->cfg.nsteps) {
    if (save_state(c, ckpt_off(c, (i + 1) / k))) return PM_ERR_CUDA;
  }
  c->next_step = i + 1;
  c->last_stepped = i;
  return PM_OK;
}

pm_status lens_project(pm_ctx* c, int32_t i) {
  if (!c) return PM_ERR_ARG;
  if (i < 0 || i >= c->cfg.nsteps) return PM_ERR_ARG;
  if (!c->ic_done || i != c->last_stepped || c->projected >= i) return PM_ERR_STATE;
  c->projected = i;
  if (!shell_active(c, i)) return PM_OK;
  return PM_DISPATCH(c, do_lens, c, i);
}

pm_status kappa_maps(pm_ctx* c, double* d_maps) {
  if (!c || !d_maps) return PM_ERR_ARG;
  if (!c->ic_done) return PM_ERR_STATE;
  if (launch_kappa_finalize(c, d_maps)) return PM_ERR_CUDA;
  return read_flags(c);
}

pm_status pm_vjp(pm_ctx* c, const double* d_dL_dkappa, double* d_dL_dnoise, double* h_dL_dparams) {
  if (!c || !d_dL_dkappa) return PM_ERR_ARG;
  if (c->cfg.ckpt_every <= 0) return PM_ERR_UNSUPPORTED;
  if (!c->ic_done || c->next_step != c->cfg.nsteps || c->projected != c->cfg.nsteps - 1 || c->vjp_state_lost)
    return PM_ERR_STATE;
  pm_status st = PM_DISPATCH(c, do_vjp, c, d_dL_dkappa, d_dL_dnoise, h_dL_dparams);
  c->s_at = 0;
  c->f_at = 0;
  // the reverse sweep reuses the particle arrays: the forward state is gone
  c->last_stepped = -1;
  c->vjp_state_lost = 1;
  return st;
}

pm_status pm_set_source_nz(pm_ctx* c, int32_t s, const double* h_z, const double* h_n, int32_t npts) {
  if (!c || !h_z || !h_n || s < 0 || s >= c->cfg.n_zs || npts < 2 || npts > 100000) return PM_ERR_ARG;
  if (c->projected >= 0) return PM_ERR_STATE;
  const double zmax = 1.0 / c->cfg.a_init - 1.0;
  double area = 0.0;
  for (int k = 0; k < npts; ++k) {
    if (!std::isfinite(h_z[k]) || !std::isfinite(h_n[k]) || h_n[k] < 0.0) return PM_ERR_ARG;
    if (k > 0 && !(h_z[k] > h_z[k - 1])) return PM_ERR_ARG;
    if (k > 0) area += 0.5 * (h_n[k] + h_n[k - 1]) * (h_z[k] - h_z[k - 1]);
  }
  if (!(h_z[0] > 0.0) || !(h_z[npts - 1] < zmax) || !(area > 0.0)) return PM_ERR_ARG;
  c->nz_z[s].assign(h_z, h_z + npts);
  c->nz_n[s].assign(h_n, h_n + npts);
  return cuda_status(set_nz_tables(c, s));
}

pm_status pm_jvp(pm_ctx* c, const double* d_noise, const double* d_dnoise, double* d_kappa, double* d_dkappa) {
  if (!c || !d_noise || !d_dnoise || !d_kappa || !d_dkappa) return PM_ERR_ARG;
  if (!c->cfg.jvp) return PM_ERR_UNSUPPORTED;
  pm_status st = PM_DISPATCH(c, do_jvp, c, d_noise, d_dnoise, d_kappa, d_dkappa);
  c->tan_on = 0;
  c->tan_noise = nullptr;
  return st;
}

pm_status pm_shot_noise_maps(pm_ctx* c, uint64_t seed, double* d_kappa) {
  if (!c || !d_kappa) return PM_ERR_ARG;
  // the run replaces the particle state: no simulation continues from here
  c->ic_done = 0;
  c->next_step = -1;
  c->last_stepped = -1;
  c->projected = -1;
  c->pgd_valid = 0;
  c->vjp_state_lost = 1;
  c->tan_on = 0;
  return PM_DISPATCH(c, do_shot_noise, c, seed, d_kappa);
}

pm_status pm_destroy(pm_ctx* c) {
  if (!c) return PM_ERR_ARG;
  delete c;
  return PM_OK;
}

const char* pm_strerror(pm_status s) {
  switch (s) {
    case PM_OK: return "ok";
    case PM_ERR_ARG: return "invalid argument or configuration";
    case PM_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case PM_ERR_CUDA: return "CUDA error";
    case PM_ERR_NONFINITE: return "non-finite value on the device";
    case PM_ERR_STATE: return "entry point called out of order";
    case PM_ERR_UNSUPPORTED: return "unsupported size or feature";
    case PM_ERR_TIMEOUT: return "device-side wait for a bulk copy timed out";
    default: return "unknown status";
  }
}

pm_status pm_get_particles(pm_ctx* c, double* d_x, double* d_p) {
  if (!c || (!d_x && !d_p)) return PM_ERR_ARG;
  if (!c->ic_done) return PM_ERR_STATE;
  return cuda_status(c->prec == PM_FP64 ? launch_get_particles<double>(c, d_x, d_p)
                                        : launch_get_particles<float>(c, d_x, d_p));
}

pm_status pm_set_particles(pm_ctx* c, const double* d_x, const double* d_p, int32_t next_step) {
  if (!c || !d_x || !d_p) return PM_ERR_ARG;
  if (next_step < 0 || next_step > c->cfg.nsteps) return PM_ERR_ARG;
  pm_status st = PM_DISPATCH(c, do_set_particles, c, d_x, d_p, next_step);
  if (st) return st;
  if (!c->ic_done) {
    if (cudaMemsetAsync(c->ws + c->L.maps, 0, (size_t)c->cfg.n_zs * c->cfg.map_npix * c->cfg.map_npix * 8,
                        c->stream))
      return PM_ERR_CUDA;
  }
  c->ic_done = 1;
  c->next_step = next_step;
  c->last_stepped = next_step - 1;
  c->projected = next_step - 2;
  c->vjp_state_lost = 1;  // no checkpoints of an externally set trajectory
  return PM_OK;
}

pm_status pm_get_forces(pm_ctx* c, double* d_f) {
  if (!c || !d_f) return PM_ERR_ARG;
  if (!c->ic_done) return PM_ERR_STATE;
  return PM_DISPATCH(c, do_readout, c, fmesh_at(c), d_f);
}

pm_status pm_get_pgd(pm_ctx* c, double* d_s) {
  if (!c || !d_s) return PM_ERR_ARG;
  if (!c->ic_done || !c->pgd_valid) return PM_ERR_STATE;
  return PM_DISPATCH(c, do_readout, c, smesh_at(c), d_s);
}

pm_status pm_fft_r2c(pm_ctx* c, const double* d_in, double* d_out) {
  if (!c || !d_in || !d_out) return PM_ERR_ARG;
  return PM_DISPATCH(c, do_fft, c, d_in, d_out);
}

pm_status pm_get_density(pm_ctx* c, double* d_rho) {
  if (!c || !d_rho) return PM_ERR_ARG;
  if (!c->ic_done) return PM_ERR_STATE;
  return PM_DISPATCH(c, do_density, c, d_rho);
}

pm_status pm_sync_status(pm_ctx* c) {
  if (!c) return PM_ERR_ARG;
  return read_flags(c);
}

pm_status pm_profile(pm_ctx* c, int32_t enable) {
  if (!c) return PM_ERR_ARG;
  if (cudaStreamSynchronize(c->stream)) return PM_ERR_CUDA;
  c->prof.resolve();
  c->prof.timing = enable != 0;
  return PM_OK;
}

pm_status pm_profile_read(pm_ctx* c, double* ms, int64_t* launches, double* bytes, int32_t nkinds) {
  if (!c || nkinds < 0) return PM_ERR_ARG;
  if (cudaStreamSynchronize(c->stream)) return PM_ERR_CUDA;
  c->prof.resolve();
  // the projection's PGD gathers: the mesh cells a gathering particle needs are its share
  // M^3 / N_p of the three PGD meshes (neighbouring particles share corner cells)
  unsigned long long ngath = 0;
  if (cudaMemcpyAsync(&ngath, lens_gather_count(c), sizeof(ngath), cudaMemcpyDeviceToHost, c->stream) ||
      cudaMemsetAsync(lens_gather_count(c), 0, sizeof(ngath), c->stream) || cudaStreamSynchronize(c->stream))
    return PM_ERR_CUDA;
  c->prof.bytes[KK_LENS] += (double)ngath * 3.0 * (double)c->rsz * (double)c->mesh_elems / (double)c->np;
  for (int k = 0; k < nkinds && k < KK_COUNT; ++k) {
    if (ms) ms[k] = c->prof.ms[k];
    if (launches) launches[k] = c->prof.launches[k];
    if (bytes) bytes[k] = c->prof.bytes[k];
  }
  for (int k = 0; k < KK_COUNT; ++k) {
    c->prof.ms[k] = 0.0;
    c->prof.launches[k] = 0;
    c->prof.bytes[k] = 0.0;
    c->prof.timed[k] = 0;
  }
  return PM_OK;
}

int32_t pm_kernel_kinds(void) { return KK_COUNT; }

const char* pm_kernel_name(int32_t kind) { return kernel_kind_name(kind); }

}  // extern "C"
