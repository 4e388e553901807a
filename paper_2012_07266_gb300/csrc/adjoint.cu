// Adjoint (reverse-mode) kernels of the PM lensing model.
//
// Transposes of the forward kernels, written by hand (Sec. 3: the model is
// differentiated with respect to the initial modes; Appendix A: Omega_m and
// sigma_8):
//  * CIC paint <-> readout: the cotangent of a readout is painted with the
//    cotangent as weight; the position derivative of a readout is the CIC
//    weight derivative (-1 / +1 along the axis) times the mesh values;
//  * the spectral operators (Poisson + gradient, PGD filter, LPT operators)
//    are transposed in the fused z pass with the conjugate multiplier
//    (fft_impl.cuh, k_zpass_combine);
//  * the lightcone projection's transpose follows the forward kernel step by
//    step and returns d/dx, d/dp and d/dS per particle;
//  * reductions (dot products) for sigma_8 and for the Omega_m finite
//    differences accumulate in FP64.
// All particle quantities are in force-mesh cell units, as in the forward.
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

__device__ __forceinline__ void unpack3(uint32_t c, int* i) {
  i[0] = c & 1023u;
  i[1] = (c >> 10) & 1023u;
  i[2] = c >> 20;
}

template <typename R>
__device__ __forceinline__ R interp_t(const R* __restrict__ t, int n, R hinv, R x) {
  const R u = x * hinv;
  int k = (int)u;
  if (k < 0) k = 0;
  if (k > n - 2) k = n - 2;
  const R f = u - (R)k;
  return t[k] * (R(1) - f) + t[k + 1] * f;
}

// block-wide sum of one double into *acc (one atomic per block)
__device__ __forceinline__ void block_add(double v, double* acc) {
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
  __syncthreads();
}

struct CIC {
  long long o[8];
  int valid;
};

template <typename R>
__device__ __forceinline__ void cic_offsets(const int* i, int M, long long* o) {
  const int x1 = i[0] + 1 == M ? 0 : i[0] + 1, y1 = i[1] + 1 == M ? 0 : i[1] + 1, z1 = i[2] + 1 == M ? 0 : i[2] + 1;
  const int xs[2] = {i[0], x1}, ys[2] = {i[1], y1}, zs[2] = {i[2], z1};
#pragma unroll
  for (int c = 0; c < 8; ++c) o[c] = ((long long)zs[c >> 2] * M + ys[(c >> 1) & 1]) * M + xs[c & 1];
}

// --------------------------------------------------------------- kernels
// paint three cotangent components (the transpose of a CIC readout of three
// meshes); x-adjacent corners share one vector reduction (FP32)
template <typename R>
__global__ void k_paint_weights(AdjState<R> s, const R* __restrict__ v0, const R* __restrict__ v1,
                                const R* __restrict__ v2, R* __restrict__ m0, R* __restrict__ m1,
                                R* __restrict__ m2, int M, long long np) {
  auto one = [&](long long j) {
    int i[3];
    unpack3(s.cell[j], i);
    const Corners c = corners(M, i[0], i[1], i[2]);
    const R fx = s.fx[j], fy = s.fy[j], fz = s.fz[j];
    scatter(m0, c, fx, fy, fz, v0[j]);
    scatter(m1, c, fx, fy, fz, v1[j]);
    scatter(m2, c, fx, fy, fz, v2[j]);
  };
  // two independent particles per iteration (overlapping their loads and reductions)
  const long long S = (long long)gridDim.x * blockDim.x;
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; j + S < np; j += 2 * S) {
    one(j);
    one(j + S);
  }
  if (j < np) one(j);
}

// Cotangent paint into per-cell interleaved meshes: NW = 3 components (one
// cotangent set: x, y, z, unused into the float4 mesh mA) or NW = 6 (two sets
// at the same positions: v_x, v_y, v_z, w_x into mA, w_y, w_z into the float2
// mesh mB).  Each block takes one contiguous run of PAINT_RUN (spatially
// sorted) particles; when the CIC footprint of the run fits a shared-memory
// tile of at most PAINT_TILE / NW cells, the run is accumulated in the tile
// (one plane per component) with shared-memory atomics and each non-zero tile
// cell is added to the meshes with one 16-byte (and one 8-byte) reduction;
// otherwise (sparse runs, runs across the periodic boundary) each corner of each
// particle is one such reduction.  The mesh reductions' L2 throughput bounds the
// untiled form.
constexpr int PAINT_THREADS = 256, PAINT_PPT = 2, PAINT_RUN = PAINT_THREADS * PAINT_PPT;
constexpr int PAINT_TILE = 12000;  // component-cells: 48 KB of static shared memory

__device__ __forceinline__ void red_v4(float* p, float a, float b, float d, float e) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(d), "f"(e)
               : "memory");
}
__device__ __forceinline__ void red_v2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

template <int NW>
__global__ void __launch_bounds__(PAINT_THREADS) k_paint_il(AdjState<float> s, const float* __restrict__ v,
                                                            const float* __restrict__ w, float* __restrict__ mA,
                                                            float* __restrict__ mB, int M, long long np) {
  constexpr int CAP = PAINT_TILE / NW;
  __shared__ float tile[NW][CAP];
  __shared__ unsigned box[6];  // lo x, y, z; hi x, y, z
  const long long jb = (long long)blockIdx.x * PAINT_RUN;
  const int tid = threadIdx.x;
  if (tid < 3) box[tid] = 0xffffffffu;
  else if (tid < 6) box[tid] = 0u;
  int cell[PAINT_PPT][3];
  unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
#pragma unroll
  for (int q = 0; q < PAINT_PPT; ++q) {
    const long long j = jb + q * PAINT_THREADS + tid;
    if (j < np) {
      unpack3(s.cell[j], cell[q]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = min(lo[a], (unsigned)cell[q][a]);
        hi[a] = max(hi[a], (unsigned)cell[q][a]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
    hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
  }
  if ((tid & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&box[a], lo[a]);
      atomicMax(&box[3 + a], hi[a]);
    }
  }
  __syncthreads();
  // tile extents: the run's cells plus the +1 CIC corner along each axis
  const int ex = (int)(box[3] - box[0]) + 2, ey = (int)(box[4] - box[1]) + 2, ez = (int)(box[5] - box[2]) + 2;
  const long long vol = (long long)ex * ey * ez;
  const bool tiled = vol <= CAP;
  if (tiled) {
    for (int t = tid; t < vol; t += PAINT_THREADS)
#pragma unroll
      for (int c = 0; c < NW; ++c) tile[c][t] = 0.f;
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PAINT_PPT; ++q) {
    const long long j = jb + q * PAINT_THREADS + tid;
    if (j >= np) continue;
    const float fx = s.fx[j], fy = s.fy[j], fz = s.fz[j];
    const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
    float u[NW];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = v[j + c * np];
    if constexpr (NW == 6) {
#pragma unroll
      for (int c = 0; c < 3; ++c) u[3 + c] = w[j + c * np];
    }
    const float wr[4] = {gz * gy, gz * fy, fz * gy, fz * fy};
    if (tiled) {
      const int tx = cell[q][0] - (int)box[0], ty = cell[q][1] - (int)box[1], tz = cell[q][2] - (int)box[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = ((tz + (r >> 1)) * ey + ty + (r & 1)) * ex + tx;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float wt = wr[r] * (dx ? fx : gx);
#pragma unroll
          for (int c = 0; c < NW; ++c) atomicAdd(&tile[c][row + dx], wt * u[c]);
        }
      }
    } else {
      const Corners cc = corners(M, cell[q][0], cell[q][1], cell[q][2]);
      const unsigned rows[4] = {cc.r00, cc.r01, cc.r10, cc.r11};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float wt = wr[r] * (dx ? fx : gx);
          const unsigned o = rows[r] + (dx ? cc.x1 : cc.x0);
          if constexpr (NW == 6) {
            red_v4(mA + 4ull * o, wt * u[0], wt * u[1], wt * u[2], wt * u[3]);
            red_v2(mB + 2ull * o, wt * u[4], wt * u[5]);
          } else {
            red_v4(mA + 4ull * o, wt * u[0], wt * u[1], wt * u[2], 0.f);
          }
        }
      }
    }
  }
  if (!tiled) return;
  __syncthreads();
  // flush: tile cell (x, y, z) is mesh cell box_lo + (x, y, z), periodic (the +1 corner of the
  // last cell of an axis is cell 0)
  for (int t = tid; t < vol; t += PAINT_THREADS) {
    float u[NW];
    bool any = false;
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      u[c] = tile[c][t];
      any |= u[c] != 0.f;
    }
    if (!any) continue;
    const int x = t % ex, yz = t / ex, y = yz % ey, z = yz / ey;
    int gx = (int)box[0] + x, gy = (int)box[1] + y, gz = (int)box[2] + z;
    gx -= gx >= M ? M : 0;
    gy -= gy >= M ? M : 0;
    gz -= gz >= M ? M : 0;
    const unsigned o = ((unsigned)gz * M + gy) * (unsigned)M + gx;
    if constexpr (NW == 6) {
      red_v4(mA + 4ull * o, u[0], u[1], u[2], u[3]);
      red_v2(mB + 2ull * o, u[4], u[5]);
    } else {
      red_v4(mA + 4ull * o, u[0], u[1], u[2], 0.f);
    }
  }
}

// lam_x += sum_c v_c grad readout(mesh_c) + mass grad readout(phi); optional
// dot = sum_j lamp_j . readout(mesh)(x_j).  TWO: a second transpose at the same
// positions in the same pass, + sum_c w_c grad readout(mesh2_c) (the PGD
// transpose of a lightcone step fused with the kick transpose of the next step).
// Each block takes one contiguous run of READ_RUN (spatially sorted) particles;
// when the run's CIC footprint fits a shared-memory tile of READ_TILE bytes for
// all the meshes read, the block first copies that box of every mesh into the
// tile (row segments, coalesced along x) and the particles gather from shared
// memory; otherwise (sparse runs, runs across the periodic boundary) they gather
// from global memory.  Each particle's dot term is formed in the path precision
// and accumulated in FP64.
template <typename R>
struct ReadoutMeshes {
  const R* m[3];   // meshes read and differentiated with cotangent v
  const R* v[3];
  const R* m2[3];  // TWO: second set, cotangent w
  const R* w[3];
};

constexpr int READ_THREADS = 256, READ_PPT = 4, READ_RUN = READ_THREADS * READ_PPT;
constexpr int READ_TILE = 48000;  // bytes of static shared memory

template <typename R, bool TWO>
__global__ void __launch_bounds__(READ_THREADS) k_readout_grad(AdjState<R> s, ReadoutMeshes<R> rm,
                                                               const R* __restrict__ phi, R mass,
                                                               R* __restrict__ lx, const R* __restrict__ lp,
                                                               double* dot, int M, long long np) {
  constexpr int NM = TWO ? 7 : 4;  // meshes read: m[0..2], phi, m2[0..2]
  constexpr int CAP = READ_TILE / (NM * (int)sizeof(R));
  __shared__ R tile[NM][CAP];
  __shared__ unsigned box[6];  // lo x, y, z; hi x, y, z
  const long long jb = (long long)blockIdx.x * READ_RUN;
  const int tid = threadIdx.x;
  if (tid < 3) box[tid] = 0xffffffffu;
  else if (tid < 6) box[tid] = 0u;
  unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
#pragma unroll
  for (int q = 0; q < READ_PPT; ++q) {
    const long long j = jb + q * READ_THREADS + tid;
    if (j < np) {
      int ci[3];
      unpack3(s.cell[j], ci);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = min(lo[a], (unsigned)ci[a]);
        hi[a] = max(hi[a], (unsigned)ci[a]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
    hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
  }
  if ((tid & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&box[a], lo[a]);
      atomicMax(&box[3 + a], hi[a]);
    }
  }
  __syncthreads();
  const int ex = (int)(box[3] - box[0]) + 2, ey = (int)(box[4] - box[1]) + 2, ez = (int)(box[5] - box[2]) + 2;
  const long long vol = (long long)ex * ey * ez;
  const bool tiled = vol <= CAP;
  // mesh mi (compile-time after unrolling): m[0..2], phi, m2[0..2]
  auto src = [&](int mi) -> const R* {
    return mi < 3 ? rm.m[mi] : mi == 3 ? phi : rm.m2[mi - 4];
  };
  if (tiled) {
    // tile cell (x, y, z) holds mesh cell box_lo + (x, y, z), periodic
    for (int t = tid; t < vol; t += READ_THREADS) {
      const int x = t % ex, yz = t / ex, y = yz % ey, z = yz / ey;
      int gx = (int)box[0] + x, gy = (int)box[1] + y, gz = (int)box[2] + z;
      gx -= gx >= M ? M : 0;
      gy -= gy >= M ? M : 0;
      gz -= gz >= M ? M : 0;
      const unsigned o = ((unsigned)gz * M + gy) * (unsigned)M + gx;
#pragma unroll
      for (int mi = 0; mi < NM; ++mi) tile[mi][t] = src(mi)[o];
    }
    __syncthreads();
  }
  double dsum = 0.0;
#pragma unroll 1
  for (int q = 0; q < READ_PPT; ++q) {
    const long long j = jb + q * READ_THREADS + tid;
    if (j >= np) continue;
    int ci[3];
    unpack3(s.cell[j], ci);  // read again: a runtime-indexed per-thread array would sit in local memory
    const R f[3] = {s.fx[j], s.fy[j], s.fz[j]};
    // corner k = (dx, dy, dz) = (k & 1, k >> 1 & 1, k >> 2): its offset in the tile or the mesh
    unsigned o[8];
    if (tiled) {
      const int tx = ci[0] - (int)box[0], ty = ci[1] - (int)box[1], tz = ci[2] - (int)box[2];
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = ((tz + (k >> 2)) * ey + ty + ((k >> 1) & 1)) * ex + tx + (k & 1);
    } else {
      const Corners cc = corners(M, ci[0], ci[1], ci[2]);
      o[0] = cc.r00 + cc.x0; o[1] = cc.r00 + cc.x1; o[2] = cc.r01 + cc.x0; o[3] = cc.r01 + cc.x1;
      o[4] = cc.r10 + cc.x0; o[5] = cc.r10 + cc.x1; o[6] = cc.r11 + cc.x0; o[7] = cc.r11 + cc.x1;
    }
    auto at = [&](int mi, int k) -> R { return tiled ? tile[mi][o[k]] : src(mi)[o[k]]; };
    const R v[3] = {rm.v[0][j], rm.v[1][j], rm.v[2][j]};
    R w[3] = {R(0), R(0), R(0)};
    if constexpr (TWO) {
#pragma unroll
      for (int c = 0; c < 3; ++c) w[c] = rm.w[c][j];
    }
    R g[3] = {R(0), R(0), R(0)};
    R val[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const R wx = dx ? f[0] : R(1) - f[0], wy = dy ? f[1] : R(1) - f[1], wz = dz ? f[2] : R(1) - f[2];
      const R sx = dx ? R(1) : R(-1), sy = dy ? R(1) : R(-1), sz = dz ? R(1) : R(-1);
      R qv = mass * at(3, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R mv = at(c, k);
        qv += v[c] * mv;
        val[c] += wx * wy * wz * mv;
        if constexpr (TWO) qv += w[c] * at(4 + c, k);
      }
      g[0] += sx * wy * wz * qv;
      g[1] += wx * sy * wz * qv;
      g[2] += wx * wy * sz * qv;
    }
    lx[j] += g[0];
    lx[j + np] += g[1];
    lx[j + 2 * np] += g[2];
    if (lp) dsum += (double)(lp[j] * val[0] + lp[j + np] * val[1] + lp[j + 2 * np] * val[2]);
  }
  if (dot) block_add(dsum, dot);
}

template <typename R>
__global__ void k_axpy(R* __restrict__ y, const R* __restrict__ x, R a, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    y[j] += a * x[j];
}

template <typename R>
__global__ void k_scale(R* __restrict__ y, const R* __restrict__ x, R a, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    y[j] = a * x[j];
}

// sum_j a_j b_j accumulated in FP64.  FP32 path: products summed in groups of up to 8 in
// FP32, one FP64 addition per group (FP64 arithmetic runs at a small fraction of the FP32
// rate on this GPU; 8 FP32 terms keep ~1e-7 relative rounding per group)
template <typename R>
__global__ void k_dot(const R* __restrict__ a, const R* __restrict__ b, long long n, double* acc) {
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    while (j < n) {
      R g = R(0);
#pragma unroll
      for (int q = 0; q < 8; ++q, j += stride)
        if (j < n) g += a[j] * b[j];
      s += (double)g;
    }
  } else {
    for (; j < n; j += stride) s += a[j] * b[j];
  }
  block_add(s, acc);
}

__global__ void k_dsum(const double* __restrict__ a, long long n, double* acc) {
  double s = 0.0;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    s += a[j];
  block_add(s, acc);
}

// out_c = scale * (ca * lam_x_c + cb * lam_p_c) on the lattice (particle j = lattice j)
template <typename R>
__global__ void k_combine2(const R* __restrict__ lx, const R* __restrict__ lp, R* __restrict__ o0,
                           R* __restrict__ o1, R* __restrict__ o2, double ca, double cb, double scale, long long n) {
  R* outs[3] = {o0, o1, o2};
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 3; ++c) outs[c][j] = (R)(scale * (ca * (double)lx[j + c * n] + cb * (double)lp[j + c * n]));
}

// sum_j lam_x . (M/L)(d1 psi1 + d2 psi2) + lam_p . (M/L)(g1 psi1 + g2 psi2)
template <typename R>
__global__ void k_ic_dot(const R* __restrict__ lx, const R* __restrict__ lp, const R* __restrict__ a0,
                         const R* __restrict__ a1, const R* __restrict__ a2, const R* __restrict__ b0,
                         const R* __restrict__ b1, const R* __restrict__ b2, double d1, double d2, double g1,
                         double g2, double cpl, long long n, double* acc) {
  double s = 0.0;
  const R* A[3] = {a0, a1, a2};
  const R* B[3] = {b0, b1, b2};
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double p1 = A[c][j], p2 = B[c] ? (double)B[c][j] : 0.0;
      s += cpl * ((double)lx[j + c * n] * (d1 * p1 + d2 * p2) + (double)lp[j + c * n] * (g1 * p1 + g2 * p2));
    }
  block_add(s, acc);
}

// cotangents of the six second-derivative fields of the 2LPT source
template <typename R>
__global__ void k_lpt2_src_adj(const R* __restrict__ ls, const R* __restrict__ d00, const R* __restrict__ d11,
                               const R* __restrict__ d22, const R* __restrict__ d01, const R* __restrict__ d02,
                               const R* __restrict__ d12, R* __restrict__ o00, R* __restrict__ o11,
                               R* __restrict__ o22, R* __restrict__ o01, R* __restrict__ o02, R* __restrict__ o12,
                               long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const R l = ls[j];
    o00[j] = l * (d11[j] + d22[j]);
    o11[j] = l * (d00[j] + d22[j]);
    o22[j] = l * (d00[j] + d11[j]);
    o01[j] = R(-2) * l * d01[j];
    o02[j] = R(-2) * l * d02[j];
    o12[j] = R(-2) * l * d12[j];
  }
}

// Transpose of the lightcone projection of one shell (mirrors k_lens).
// Adds d/dx, d/dp (cells) to lam_x, lam_p and writes d/dS (cells) to vS.
// Three resident blocks per SM (80 registers in FP32, no spills): the kernel
// waits on its gathers, so resident warps beat registers (93 vs 102 ms per
// 256^3 adjoint).
template <typename R>
__global__ void __launch_bounds__(256, 3) k_lens_vjp(const LensAdjArgs<R> A) {
  const R cell_len = A.g.cell_len;
  const R fov_half = A.g.fov_half, inv_dth = A.g.inv_dtheta;
  const R tan_half = A.g.tan_half, margin = A.g.margin;
  // whole warps iterate together (warp-level replica culling, as in the forward)
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); j0 < A.np; j0 += stride) {
    const bool valid = j0 + lane < A.np;
    const long long j = valid ? j0 + lane : A.np - 1;
    int ci[3];
    unpack3(A.st.cell[j], ci);
    const R cf[3] = {A.st.fx[j], A.st.fy[j], A.st.fz[j]};
    const R cp[3] = {A.st.px[j], A.st.py[j], A.st.pz[j]};
    R cs[3] = {R(0), R(0), R(0)};
    bool have_s = false;
    R gx[3] = {0, 0, 0}, gp[3] = {0, 0, 0}, gs[3] = {0, 0, 0};
    const WarpBox box =
        warp_box(valid, (float)ci[0] + (float)cf[0], (float)ci[1] + (float)cf[1], (float)ci[2] + (float)cf[2]);
    // the particle's PGD displacement (cells), CIC-gathered from the three PGD meshes
    auto gather_s = [&]() {
      const R* Sm[3] = {A.S0, A.S1, A.S2};
      long long o[8];
      cic_offsets<R>(ci, A.M, o);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          acc += ((k & 1) ? cf[0] : R(1) - cf[0]) * (((k >> 1) & 1) ? cf[1] : R(1) - cf[1]) *
                 ((k >> 2) ? cf[2] : R(1) - cf[2]) * Sm[c][o[k]];
        cs[c] = acc;
      }
      have_s = true;
    };
    // one replica of this particle (the per-particle tests below decide exactly)
    auto project = [&](int q) {
      const Replica rp = A.rep[q];
      R r[3], gf[3];
      int gi[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int ax = rp.perm[d];
        int i = pick3(ax, ci[0], ci[1], ci[2]);
        R f = pick3(ax, cf[0], cf[1], cf[2]);
        if (rp.flip >> d & 1) {
          if (f > R(0)) { i = A.M - 1 - i; f = R(1) - f; }
          else { i = i == 0 ? 0 : A.M - i; }
        }
        i += rp.shift[d];
        if (i >= A.M) i -= A.M;
        gi[d] = i + rp.n[d] * A.M;
        gf[d] = f;
        r[d] = ((R)gi[d] + f) * cell_len;
      }
      const R chi2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (!(r[2] > R(0) && in_shell<R>(chi2, gi, gf, A.cell_len, A.chi_lo2, A.chi_hi2, A.g.lo2, A.g.hi2))) return;
      const R lim = r[2] * tan_half + margin;
      if (fabs(r[0]) > lim || fabs(r[1]) > lim) return;
      if (A.S0 && !have_s) gather_s();
      R pr[3], sr[3], sg[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        sg[d] = (rp.flip >> d & 1) ? R(-1) : R(1);
        pr[d] = sg[d] * pick3((int)rp.perm[d], cp[0], cp[1], cp[2]);
        sr[d] = sg[d] * pick3((int)rp.perm[d], cs[0], cs[1], cs[2]);
      }
      const R chi = sqrt(chi2);
      R rc[3] = {r[0], r[1], r[2]};
      R dt = R(0), ddt = R(0);
      if (A.sub) {
        const R t = interp_t<R>(A.tab_d1, A.tab_n, A.g.tab_hinv, chi);
        dt = (t - A.d1_next_r) * A.inv_gp_half_r;
        ddt = interp_t<R>(A.tab_dd1, A.tab_n, A.g.tab_hinv, chi) * A.inv_gp_half_r;
#pragma unroll
        for (int d = 0; d < 3; ++d) rc[d] += pr[d] * dt * cell_len;
      }
      if (A.S0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) rc[d] += sr[d] * cell_len;
      }
      if (!(rc[2] > R(0))) return;
      const R chic = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
      const R inz = R(1) / rc[2];
      const R u = (rc[0] * inz + fov_half) * inv_dth - R(0.5);
      const R v = (rc[1] * inz + fov_half) * inv_dth - R(0.5);
      if (!isfinite(u) || !isfinite(v)) return;
      if (u < R(-1) || v < R(-1) || u >= (R)A.npix || v >= (R)A.npix) return;
      const R fu0 = floor(u), fv0 = floor(v);
      const int iu = (int)fu0, iv = (int)fv0;
      const R fu = u - fu0, fv = v - fv0;
      const R cd = chic;
      const R inva = interp_t<R>(A.tab_inva, A.tab_n, A.g.tab_hinv, cd);
      const R dinva = interp_t<R>(A.tab_dinva, A.tab_n, A.g.tab_hinv, cd);
      R grc[3] = {0, 0, 0};
      for (int s = 0; s < A.nzs; ++s) {
        R w, dw;
        if (A.nz_mask >> s & 1u) {
          // source distribution: w = wpref q / (chi a), dw/dchi from q and dq/dchi
          const R qv = interp_t<R>(A.qtab + (size_t)s * A.tab_n, A.tab_n, A.g.tab_hinv, cd);
          if (!(qv > R(0))) continue;
          const R dqv = interp_t<R>(A.dqtab + (size_t)s * A.tab_n, A.tab_n, A.g.tab_hinv, cd);
          w = A.wpref_r * qv / cd * inva;
          dw = A.wpref_r * ((dqv * cd - qv) / (cd * cd) * inva + qv / cd * dinva);
        } else {
          const R csd = A.chi_s_r[s];
          if (!(cd < csd)) continue;
          const R fr = R(1) / cd - R(1) / csd;
          w = A.wpref_r * fr * inva;
          dw = A.wpref_r * (-inva / (cd * cd) + fr * dinva);
        }
        const R* lam = A.lam + s * A.npix * A.npix;
        R Lw = 0, Lu = 0, Lv = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int du = k & 1, dv = k >> 1;
          const int jx = iu + du, jy = iv + dv;
          if (jx < 0 || jx >= A.npix || jy < 0 || jy >= A.npix) continue;
          const R l = lam[jy * A.npix + jx];
          const R wu = du ? fu : R(1) - fu, wv = dv ? fv : R(1) - fv;
          Lw += l * wu * wv;
          Lu += l * (du ? R(1) : R(-1)) * wv;
          Lv += l * wu * (dv ? R(1) : R(-1));
        }
        const R rad = dw * Lw / cd;
        const R gu = w * Lu * inv_dth, gv = w * Lv * inv_dth;
        grc[0] += rad * rc[0] + gu / rc[2];
        grc[1] += rad * rc[1] + gv / rc[2];
        grc[2] += rad * rc[2] - (gu * rc[0] + gv * rc[1]) / (rc[2] * rc[2]);
      }
      // rc = r + pr dt(|r|) L_cell + sr L_cell
      R gr[3] = {grc[0], grc[1], grc[2]};
      if (A.sub) {
        const R gdp = (grc[0] * pr[0] + grc[1] * pr[1] + grc[2] * pr[2]) * cell_len * ddt / chi;
#pragma unroll
        for (int d = 0; d < 3; ++d) gr[d] += gdp * r[d];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int ax = rp.perm[d];
        const R vx = sg[d] * gr[d] * cell_len, vs = sg[d] * grc[d] * cell_len;
        const R vp = A.sub ? vs * dt : R(0);
        // scatter to the particle's own axis ax with constant indices (no local memory)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const bool hit = a == ax;
          gx[a] += hit ? vx : R(0);
          gp[a] += hit ? vp : R(0);
          gs[a] += hit ? vs : R(0);
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
    if (!valid) continue;
    A.lx[j] += gx[0];
    A.lx[j + A.np] += gx[1];
    A.lx[j + 2 * A.np] += gx[2];
    A.lp[j] += gp[0];
    A.lp[j + A.np] += gp[1];
    A.lp[j + 2 * A.np] += gp[2];
    if (A.vS) {
      A.vS[j] += gs[0];
      A.vS[j + A.np] += gs[1];
      A.vS[j + 2 * A.np] += gs[2];
    }
  }
}

}  // namespace

// -------------------------------------------------------------- launchers
static int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 16);
}

template <typename R>
void adj_paint_weights(const AdjState<R>& s, const R* v, R* const* meshes, int M, long long np, cudaStream_t st,
                       Prof* pf) {
  ProfScope ps(pf, KK_ADJ_PAINT, st, np * (4.0 + 6.0 * sizeof(R)) + 3.0 * (double)M * M * M * sizeof(R));
  k_paint_weights<R><<<blocks_for(np), 256, 0, st>>>(s, v, v + np, v + 2 * np, meshes[0], meshes[1], meshes[2], M, np);
}

void adj_paint_weights4(const AdjState<float>& s, const float* v, float* mesh4, int M, long long np, cudaStream_t st,
                        Prof* pf) {
  ProfScope ps(pf, KK_ADJ_PAINT, st, np * (4.0 + 6.0 * sizeof(float)) + 4.0 * (double)M * M * M * sizeof(float));
  const long long nb = (np + PAINT_RUN - 1) / PAINT_RUN;
  if (nb > 0) k_paint_il<3><<<(unsigned)nb, PAINT_THREADS, 0, st>>>(s, v, nullptr, mesh4, nullptr, M, np);
}

void adj_paint_weights6(const AdjState<float>& s, const float* v, const float* w, float* mesh4, float* mesh2, int M,
                        long long np, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ_PAINT, st, np * (4.0 + 9.0 * sizeof(float)) + 6.0 * (double)M * M * M * sizeof(float));
  const long long nb = (np + PAINT_RUN - 1) / PAINT_RUN;
  if (nb > 0) k_paint_il<6><<<(unsigned)nb, PAINT_THREADS, 0, st>>>(s, v, w, mesh4, mesh2, M, np);
}

template <typename R>
void adj_readout_grad(const AdjState<R>& s, R* const* meshes, const R* v, const R* phi, double mass, R* lx,
                      const R* lp, double* dot, int M, long long np, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ_READ, st, np * (4.0 + 12.0 * sizeof(R)) + 4.0 * (double)M * M * M * sizeof(R));
  ReadoutMeshes<R> rm = {};
  for (int c = 0; c < 3; ++c) {
    rm.m[c] = meshes[c];
    rm.v[c] = v + c * np;
  }
  const long long nb = (np + READ_RUN - 1) / READ_RUN;
  if (nb > 0) k_readout_grad<R, false><<<(unsigned)nb, READ_THREADS, 0, st>>>(s, rm, phi, (R)mass, lx, lp, dot, M, np);
}

template <typename R>
void adj_readout_grad2(const AdjState<R>& s, R* const* meshes, const R* v, R* const* meshes2, const R* w,
                       const R* phi, double mass, R* lx, const R* lp, double* dot, int M, long long np, cudaStream_t st,
                       Prof* pf) {
  ProfScope ps(pf, KK_ADJ_READ, st, np * (4.0 + 18.0 * sizeof(R)) + 7.0 * (double)M * M * M * sizeof(R));
  ReadoutMeshes<R> rm;
  for (int c = 0; c < 3; ++c) {
    rm.m[c] = meshes[c];
    rm.v[c] = v + c * np;
    rm.m2[c] = meshes2[c];
    rm.w[c] = w + c * np;
  }
  const long long nb = (np + READ_RUN - 1) / READ_RUN;
  if (nb > 0) k_readout_grad<R, true><<<(unsigned)nb, READ_THREADS, 0, st>>>(s, rm, phi, (R)mass, lx, lp, dot, M, np);
}

template <typename R>
void adj_axpy(R* y, const R* x, double a, long long n, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 3.0 * n * sizeof(R));
  k_axpy<R><<<blocks_for(n), 256, 0, st>>>(y, x, (R)a, n);
}

template <typename R>
void adj_scale(R* y, const R* x, double a, long long n, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 2.0 * n * sizeof(R));
  k_scale<R><<<blocks_for(n), 256, 0, st>>>(y, x, (R)a, n);
}

template <typename R>
void adj_dot(const R* a, const R* b, long long n, double* acc, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 2.0 * n * sizeof(R));
  k_dot<R><<<blocks_for(n), 256, 0, st>>>(a, b, n, acc);
}

void adj_dsum(const double* a, long long n, double* acc, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 8.0 * n);
  k_dsum<<<blocks_for(n), 256, 0, st>>>(a, n, acc);
}

template <typename R>
void adj_combine2(const R* lx, const R* lp, R* const* outs, double ca, double cb, double scale, long long n,
                  cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 9.0 * n * sizeof(R));
  k_combine2<R><<<blocks_for(n), 256, 0, st>>>(lx, lp, outs[0], outs[1], outs[2], ca, cb, scale, n);
}

template <typename R>
void adj_ic_dot(const R* lx, const R* lp, R* const* psi1, R* const* psi2, double d1, double d2, double g1, double g2,
                double cpl, long long n, double* acc, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 12.0 * n * sizeof(R));
  k_ic_dot<R><<<blocks_for(n), 256, 0, st>>>(lx, lp, psi1[0], psi1[1], psi1[2], psi2 ? psi2[0] : nullptr,
                                             psi2 ? psi2[1] : nullptr, psi2 ? psi2[2] : nullptr, d1, d2, g1, g2, cpl,
                                             n, acc);
}

template <typename R>
void adj_lpt2_src(const R* ls, R* const* d, R* const* out, long long n, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ, st, 13.0 * n * sizeof(R));
  k_lpt2_src_adj<R><<<blocks_for(n), 256, 0, st>>>(ls, d[0], d[1], d[2], d[3], d[4], d[5], out[0], out[1], out[2],
                                                   out[3], out[4], out[5], n);
}

template <typename R>
void adj_lens(const LensAdjArgs<R>& A, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, KK_ADJ_LENS, st, A.np * (4.0 + 12.0 * sizeof(R)));
  k_lens_vjp<R><<<(int)std::min<long long>((A.np + 255) / 256, 152LL * 8), 256, 0, st>>>(A);
}

#define PM_ADJ_INST(R)                                                                                          \
  template void adj_paint_weights<R>(const AdjState<R>&, const R*, R* const*, int, long long, cudaStream_t,     \
                                     Prof*);                                                                    \
  template void adj_readout_grad<R>(const AdjState<R>&, R* const*, const R*, const R*, double, R*, const R*,    \
                                    double*, int, long long, cudaStream_t, Prof*);                              \
  template void adj_readout_grad2<R>(const AdjState<R>&, R* const*, const R*, R* const*, const R*, const R*,    \
                                     double, R*, const R*, double*, int, long long, cudaStream_t, Prof*);       \
  template void adj_axpy<R>(R*, const R*, double, long long, cudaStream_t, Prof*);                              \
  template void adj_scale<R>(R*, const R*, double, long long, cudaStream_t, Prof*);                             \
  template void adj_dot<R>(const R*, const R*, long long, double*, cudaStream_t, Prof*);                        \
  template void adj_combine2<R>(const R*, const R*, R* const*, double, double, double, long long, cudaStream_t, \
                                Prof*);                                                                         \
  template void adj_ic_dot<R>(const R*, const R*, R* const*, R* const*, double, double, double, double, double, \
                              long long, double*, cudaStream_t, Prof*);                                         \
  template void adj_lpt2_src<R>(const R*, R* const*, R* const*, long long, cudaStream_t, Prof*);                \
  template void adj_lens<R>(const LensAdjArgs<R>&, cudaStream_t, Prof*);
PM_ADJ_INST(float)
PM_ADJ_INST(double)

}  // namespace pmlens
