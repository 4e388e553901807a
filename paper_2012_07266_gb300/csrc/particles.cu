// Particle kernels: LPT initial positions, cloud-in-cell paint, the fused
// kick + drift + paint of a FastPM step, CIC readout, state transfer.
//
// Particle state (structure of arrays, HBM resident): a packed uint32 cell
// index (ix | iy << 10 | iz << 20, force-mesh cells, mesh <= 1024) and the
// in-cell fraction f in [0, 1) per axis, so that the position is (i + f) cells;
// momentum in cell units.  Positions keep ~2^-24 cell precision everywhere in
// the box with FP32 fractions.
#include <algorithm>
#include <cmath>

#include "cic.cuh"
#include "pm_internal.h"

namespace pmlens {

namespace {

__device__ __forceinline__ void unpack(uint32_t c, int& ix, int& iy, int& iz) {
  ix = c & 1023u;
  iy = (c >> 10) & 1023u;
  iz = c >> 20;
}
__device__ __forceinline__ uint32_t pack(int ix, int iy, int iz) {
  return (uint32_t)ix | ((uint32_t)iy << 10) | ((uint32_t)iz << 20);
}
__device__ __forceinline__ int wrapi(long long i, int M) {
  long long r = i % M;
  return (int)(r < 0 ? r + M : r);
}
// 32-bit wrap for the per-step carry (|i| far below 2^31)
__device__ __forceinline__ int wrap32(int i, int M) {
  int r = i % M;
  return r < 0 ? r + M : r;
}

// split a coordinate in cells into (wrapped integer cell, fraction in [0,1))
template <typename R>
__device__ __forceinline__ void split_cells(double X, int M, int& i, R& f) {
  const double fl = floor(X);
  R fr = (R)(X - fl);
  long long ii = (long long)fl;
  if (fr >= R(1)) { fr = R(0); ii += 1; }
  i = wrapi(ii, M);
  f = fr;
}

template <typename R>
struct PState {
  uint32_t* cell;
  R *fx, *fy, *fz, *px, *py, *pz;
};

template <typename R>
PState<R> pstate(pm_ctx* c) {
  PState<R> s;
  s.cell = reinterpret_cast<uint32_t*>(c->ws + c->L.cell);
  R* f = reinterpret_cast<R*>(c->ws + c->L.frac);
  R* p = reinterpret_cast<R*>(c->ws + c->L.mom);
  s.fx = f; s.fy = f + c->np; s.fz = f + 2 * c->np;
  s.px = p; s.py = p + c->np; s.pz = p + 2 * c->np;
  return s;
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = 152LL * 16;
  return (int)(b < cap ? b : cap);
}

// ------------------------------------------------------------------ kernels
template <typename R>
__global__ void k_ic_particles(PState<R> s, const R* __restrict__ p1x, const R* __restrict__ p1y,
                               const R* __restrict__ p1z, const R* __restrict__ p2x, const R* __restrict__ p2y,
                               const R* __restrict__ p2z, int nc, int M, double cell_per_len, double d1,
                               double d2, double gp1, double gp2, long long np) {
  const double lat = (double)M / (double)nc;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    const int jx = (int)(j % nc), jy = (int)((j / nc) % nc), jz = (int)(j / ((long long)nc * nc));
    double sx = p1x[j], sy = p1y[j], sz = p1z[j];
    double tx = 0, ty = 0, tz = 0;
    if (p2x) { tx = p2x[j]; ty = p2y[j]; tz = p2z[j]; }
    int ix, iy, iz;
    R fx, fy, fz;
    split_cells<R>(jx * lat + 0.5 + (d1 * sx + d2 * tx) * cell_per_len, M, ix, fx);
    split_cells<R>(jy * lat + 0.5 + (d1 * sy + d2 * ty) * cell_per_len, M, iy, fy);
    split_cells<R>(jz * lat + 0.5 + (d1 * sz + d2 * tz) * cell_per_len, M, iz, fz);
    s.cell[j] = pack(ix, iy, iz);
    s.fx[j] = fx; s.fy[j] = fy; s.fz[j] = fz;
    s.px[j] = (R)((gp1 * sx + gp2 * tx) * cell_per_len);
    s.py[j] = (R)((gp1 * sy + gp2 * ty) * cell_per_len);
    s.pz[j] = (R)((gp1 * sz + gp2 * tz) * cell_per_len);
  }
}

// CIC paint.  The state is kept sorted by coarse spatial bucket, so the
// reductions of a warp hit few L2 lines; plain (vector) reductions measured
// faster than warp-aggregating same-cell lanes first.
template <typename R>
__global__ void __launch_bounds__(256) k_paint(PState<R> s, R* __restrict__ rho, int M, R mass, long long np) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    unpack(s.cell[j], ix, iy, iz);
    scatter(rho, corners(M, ix, iy, iz), s.fx[j], s.fy[j], s.fz[j], mass);
  }
}

// kick with the force at the current position, drift, paint the new position
template <typename R>
__device__ __forceinline__ void kdk_one(PState<R> s, const R* __restrict__ F0, const R* __restrict__ F1,
                                        const R* __restrict__ F2, R* __restrict__ rho, int M, R ckick, R cdrift,
                                        R mass, long long j) {
  int ix, iy, iz;
  unpack(s.cell[j], ix, iy, iz);
  R fx = s.fx[j], fy = s.fy[j], fz = s.fz[j];
  const Corners c = corners(M, ix, iy, iz);
  const R px = s.px[j] + ckick * gather(F0, c, fx, fy, fz);
  const R py = s.py[j] + ckick * gather(F1, c, fx, fy, fz);
  const R pz = s.pz[j] + ckick * gather(F2, c, fx, fy, fz);
  // drift in cell units; carry the integer part into the cell index
  R nx = fx + px * cdrift, ny = fy + py * cdrift, nz = fz + pz * cdrift;
  R cx = floor(nx), cy = floor(ny), cz = floor(nz);
  nx -= cx; ny -= cy; nz -= cz;
  if (nx >= R(1)) { nx -= R(1); cx += R(1); }
  if (ny >= R(1)) { ny -= R(1); cy += R(1); }
  if (nz >= R(1)) { nz -= R(1); cz += R(1); }
  ix = wrap32(ix + (int)cx, M);
  iy = wrap32(iy + (int)cy, M);
  iz = wrap32(iz + (int)cz, M);
  s.px[j] = px; s.py[j] = py; s.pz[j] = pz;
  s.cell[j] = pack(ix, iy, iz);
  s.fx[j] = nx; s.fy[j] = ny; s.fz[j] = nz;
  scatter(rho, corners(M, ix, iy, iz), nx, ny, nz, mass);
}

template <typename R>
__global__ void __launch_bounds__(256) k_kdk_paint(PState<R> s, const R* __restrict__ F0, const R* __restrict__ F1,
                                                   const R* __restrict__ F2, R* __restrict__ rho, int M, R ckick,
                                                   R cdrift, R mass, long long np) {
  // each block walks one contiguous run of the (spatially sorted) particles, so that the mesh
  // rows its gathers and reductions touch are reused while they are in L2; two independent
  // particles per thread and iteration (adjacent lines): their gathers and reductions overlap
  const long long per = (np + gridDim.x - 1) / gridDim.x;
  const long long j0 = blockIdx.x * per, j1 = j0 + per < np ? j0 + per : np;
  for (long long j = j0 + threadIdx.x; j < j1; j += 2 * (long long)blockDim.x) {
    kdk_one(s, F0, F1, F2, rho, M, ckick, cdrift, mass, j);
    if (j + blockDim.x < j1) kdk_one(s, F0, F1, F2, rho, M, ckick, cdrift, mass, j + blockDim.x);
  }
}

// readout at the particles, written in lattice order (out[pid[j]])
template <typename R>
__global__ void k_readout(PState<R> s, const uint32_t* __restrict__ pid, const R* __restrict__ m0,
                          const R* __restrict__ m1, const R* __restrict__ m2, int M, double scale,
                          double* __restrict__ out, long long np) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    unpack(s.cell[j], ix, iy, iz);
    const Corners c = corners(M, ix, iy, iz);
    const R fx = s.fx[j], fy = s.fy[j], fz = s.fz[j];
    const long long o = pid[j];
    out[3 * o + 0] = scale * (double)gather(m0, c, fx, fy, fz);
    out[3 * o + 1] = scale * (double)gather(m1, c, fx, fy, fz);
    out[3 * o + 2] = scale * (double)gather(m2, c, fx, fy, fz);
  }
}

template <typename R>
__global__ void k_set_particles(PState<R> s, const double* __restrict__ x, const double* __restrict__ p, int M,
                                double cell_per_len, long long np) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    R fx, fy, fz;
    split_cells<R>(x[3 * j + 0] * cell_per_len, M, ix, fx);
    split_cells<R>(x[3 * j + 1] * cell_per_len, M, iy, fy);
    split_cells<R>(x[3 * j + 2] * cell_per_len, M, iz, fz);
    s.cell[j] = pack(ix, iy, iz);
    s.fx[j] = fx; s.fy[j] = fy; s.fz[j] = fz;
    s.px[j] = (R)(p[3 * j + 0] * cell_per_len);
    s.py[j] = (R)(p[3 * j + 1] * cell_per_len);
    s.pz[j] = (R)(p[3 * j + 2] * cell_per_len);
  }
}

// Uniformly random particles for a shot-noise run (Sec. 4): coordinate k of
// particle j is output 3j + k of SplitMix64 seeded with `seed` (the state
// seed + (n + 1) * gamma, mixed), whose top 24 bits r place it at
// r M / 2^24 cells: integer cell (r M) >> 24 and the exact fraction of the
// low 24 bits.  Zero momentum.
template <typename R>
__global__ void k_random_particles(PState<R> s, uint64_t seed, int M, long long np) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    R f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint64_t z = seed + (uint64_t)(3 * j + k + 1) * 0x9E3779B97F4A7C15ULL;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
      z ^= z >> 31;
      const uint64_t t = (z >> 40) * (uint64_t)M;
      ci[k] = (int)(t >> 24);
      f[k] = (R)((double)(t & 0xFFFFFFu) * 0x1p-24);
    }
    s.cell[j] = pack(ci[0], ci[1], ci[2]);
    s.fx[j] = f[0]; s.fy[j] = f[1]; s.fz[j] = f[2];
    s.px[j] = (R)0; s.py[j] = (R)0; s.pz[j] = (R)0;
  }
}

template <typename R>
__global__ void k_get_particles(PState<R> s, const uint32_t* __restrict__ pid, double* __restrict__ x,
                                double* __restrict__ p, double len_per_cell, long long np) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < np; j += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    unpack(s.cell[j], ix, iy, iz);
    const long long o = pid[j];  // lattice order
    if (x) {
      x[3 * o + 0] = ((double)ix + (double)s.fx[j]) * len_per_cell;
      x[3 * o + 1] = ((double)iy + (double)s.fy[j]) * len_per_cell;
      x[3 * o + 2] = ((double)iz + (double)s.fz[j]) * len_per_cell;
    }
    if (p) {
      p[3 * o + 0] = (double)s.px[j] * len_per_cell;
      p[3 * o + 1] = (double)s.py[j] * len_per_cell;
      p[3 * o + 2] = (double)s.pz[j] * len_per_cell;
    }
  }
}

template <typename R>
__global__ void k_lpt2_source(const R* __restrict__ d00, const R* __restrict__ d11, const R* __restrict__ d22,
                              const R* __restrict__ d01, const R* __restrict__ d02, const R* __restrict__ d12,
                              R* __restrict__ src, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const R a = d00[j], b = d11[j], c = d22[j], e = d01[j], f = d02[j], g = d12[j];
    src[j] = a * b + a * c + b * c - e * e - f * f - g * g;
  }
}

template <typename R>
__global__ void k_convert_in(const double* __restrict__ in, R* __restrict__ out, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    out[j] = (R)in[j];
}

template <typename R>
__global__ void k_convert_out(const R* __restrict__ in, double* __restrict__ out, long long n, double scale) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    out[j] = scale * (double)in[j];
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename R>
cudaError_t launch_ic_particles(pm_ctx* c, R* const* psi1, R* const* psi2, double d1, double d2, double gp1,
                                double gp2) {
  const double cpl = c->M / c->cfg.box;
  ProfScope ps(&c->prof, KK_IC, c->stream);
  k_ic_particles<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(
      pstate<R>(c), psi1[0], psi1[1], psi1[2], psi2 ? psi2[0] : nullptr, psi2 ? psi2[1] : nullptr,
      psi2 ? psi2[2] : nullptr, c->nc, c->M, cpl, d1, d2, gp1, gp2, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_paint(pm_ctx* c, R* rho) {
  const double mass = std::pow((double)c->M / c->nc, 3.0);
  ProfScope ps(&c->prof, KK_PAINT, c->stream, c->np * (4.0 + 3.0 * sizeof(R)) + c->mesh_elems * (double)sizeof(R));
  k_paint<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(pstate<R>(c), rho, c->M, (R)mass, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_kdk_paint(pm_ctx* c, R* rho, double ckick, double cdrift) {
  const double mass = std::pow((double)c->M / c->nc, 3.0);
  R* F = reinterpret_cast<R*>(c->ws + fmesh_at(c));  // F(x_i)
  // state read + written, three force meshes gathered, density written
  ProfScope ps(&c->prof, KK_KDK_PAINT, c->stream,
               2.0 * c->np * (4.0 + 6.0 * sizeof(R)) + 4.0 * c->mesh_elems * (double)sizeof(R));
  // up to 64 blocks' worth per SM, so that each block's run of sorted particles is short (~1700
  // at 256^3): 1.013 -> 0.882 ms per pm256 launch against 16 per SM (longer runs keep more of
  // the mesh in flight per block and re-fetch more of it)
  const int blocks = (int)std::min<long long>((c->np + 255) / 256, 152LL * 64);
  k_kdk_paint<R><<<blocks, 256, 0, c->stream>>>(pstate<R>(c), F, F + c->mesh_elems,
                                                               F + 2 * c->mesh_elems, rho, c->M, (R)ckick,
                                                               (R)cdrift, (R)mass, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_readout(pm_ctx* c, R* const* meshes, double scale, double* out) {
  ProfScope ps(&c->prof, KK_MISC, c->stream);
  k_readout<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(
      pstate<R>(c), reinterpret_cast<const uint32_t*>(c->ws + c->L.pid), meshes[0], meshes[1], meshes[2], c->M, scale,
      out, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_set_particles(pm_ctx* c, const double* x, const double* p) {
  ProfScope ps(&c->prof, KK_MISC, c->stream);
  k_set_particles<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(pstate<R>(c), x, p, c->M, c->M / c->cfg.box,
                                                                   c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_random_particles(pm_ctx* c, uint64_t seed) {
  ProfScope ps(&c->prof, KK_IC, c->stream);
  k_random_particles<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(pstate<R>(c), seed, c->M, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_get_particles(pm_ctx* c, double* x, double* p) {
  ProfScope ps(&c->prof, KK_MISC, c->stream);
  k_get_particles<R><<<grid_for(c->np, 256), 256, 0, c->stream>>>(
      pstate<R>(c), reinterpret_cast<const uint32_t*>(c->ws + c->L.pid), x, p, c->cfg.box / c->M, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lpt2_source(pm_ctx* c, R* const* d, R* src, long long n) {
  ProfScope ps(&c->prof, KK_IC, c->stream);
  k_lpt2_source<R><<<grid_for(n, 256), 256, 0, c->stream>>>(d[0], d[1], d[2], d[3], d[4], d[5], src, n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_convert_in(const double* in, R* out, long long n, cudaStream_t s, Prof* pf) {
  ProfScope ps(pf, KK_MISC, s);
  k_convert_in<R><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_convert_out(const R* in, double* out, long long n, double scale, cudaStream_t s, Prof* pf) {
  ProfScope ps(pf, KK_MISC, s);
  k_convert_out<R><<<grid_for(n, 256), 256, 0, s>>>(in, out, n, scale);
  return cudaGetLastError();
}

#define PM_INST(R)                                                                                        \
  template cudaError_t launch_ic_particles<R>(pm_ctx*, R* const*, R* const*, double, double, double, double); \
  template cudaError_t launch_paint<R>(pm_ctx*, R*);                                                      \
  template cudaError_t launch_kdk_paint<R>(pm_ctx*, R*, double, double);                                  \
  template cudaError_t launch_readout<R>(pm_ctx*, R* const*, double, double*);                            \
  template cudaError_t launch_set_particles<R>(pm_ctx*, const double*, const double*);                    \
  template cudaError_t launch_get_particles<R>(pm_ctx*, double*, double*);                                \
  template cudaError_t launch_random_particles<R>(pm_ctx*, uint64_t);                                     \
  template cudaError_t launch_lpt2_source<R>(pm_ctx*, R* const*, R*, long long);                          \
  template cudaError_t launch_convert_in<R>(const double*, R*, long long, cudaStream_t, Prof*);            \
  template cudaError_t launch_convert_out<R>(const R*, double*, long long, double, cudaStream_t, Prof*);
PM_INST(float)
PM_INST(double)

}  // namespace pmlens
