// Cloud-in-cell corner addressing, gather and scatter shared by the forward
// particle kernels and their adjoints.  Meshes are [z][y][x] with M^3 <= 2^30
// cells, so row offsets fit 32 bits; the two x-neighbours of a corner row are
// adjacent floats and, when they share an aligned quad, move as one 16-byte
// vector reduction.
#pragma once

#include <cuda_runtime.h>

namespace pmlens {
namespace {

struct Corners {
  unsigned r00, r01, r10, r11;  // row offsets (z, y) of the 4 x-rows (M^3 <= 2^30)
  int x0, x1;
};

__device__ __forceinline__ Corners corners(int M, int ix, int iy, int iz) {
  const int ix1 = ix + 1 == M ? 0 : ix + 1;
  const int iy1 = iy + 1 == M ? 0 : iy + 1;
  const int iz1 = iz + 1 == M ? 0 : iz + 1;
  Corners c;
  c.r00 = ((unsigned)iz * M + iy) * M;
  c.r01 = ((unsigned)iz * M + iy1) * M;
  c.r10 = ((unsigned)iz1 * M + iy) * M;
  c.r11 = ((unsigned)iz1 * M + iy1) * M;
  c.x0 = ix;
  c.x1 = ix1;
  return c;
}

template <typename R>
__device__ __forceinline__ R gather(const R* __restrict__ m, const Corners& c, R fx, R fy, R fz) {
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R a = gx * __ldg(m + c.r00 + c.x0) + fx * __ldg(m + c.r00 + c.x1);
  const R b = gx * __ldg(m + c.r01 + c.x0) + fx * __ldg(m + c.r01 + c.x1);
  const R d = gx * __ldg(m + c.r10 + c.x0) + fx * __ldg(m + c.r10 + c.x1);
  const R e = gx * __ldg(m + c.r11 + c.x0) + fx * __ldg(m + c.r11 + c.x1);
  return gz * (gy * a + fy * b) + fz * (gy * d + fy * e);
}

// add (a, b) to the x-adjacent cells r[x0], r[x1] (x1 = x0 + 1 unless wrapped):
// one 16-byte vector reduction when both fall in one aligned quad of floats
__device__ __forceinline__ void red_pair(float* row, int x0, int x1, float a, float b) {
  const int q = x0 & 3;
  if (x1 == x0 + 1 && q != 3) {
    float* base = row + (x0 & ~3);
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    if (q == 0) { v0 = a; v1 = b; } else if (q == 1) { v1 = a; v2 = b; } else { v2 = a; v3 = b; }
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(base), "f"(v0), "f"(v1), "f"(v2), "f"(v3)
                 : "memory");
  } else {
    atomicAdd(row + x0, a);
    atomicAdd(row + x1, b);
  }
}

__device__ __forceinline__ void scatter(float* __restrict__ m, const Corners& c, float fx, float fy, float fz,
                                        float w) {
  const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
  const float w00 = w * gz * gy, w01 = w * gz * fy, w10 = w * fz * gy, w11 = w * fz * fy;
  red_pair(m + c.r00, c.x0, c.x1, w00 * gx, w00 * fx);
  red_pair(m + c.r01, c.x0, c.x1, w01 * gx, w01 * fx);
  red_pair(m + c.r10, c.x0, c.x1, w10 * gx, w10 * fx);
  red_pair(m + c.r11, c.x0, c.x1, w11 * gx, w11 * fx);
}

template <typename R>
__device__ __forceinline__ void scatter(R* __restrict__ m, const Corners& c, R fx, R fy, R fz, R w) {
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R w00 = w * gz * gy, w01 = w * gz * fy, w10 = w * fz * gy, w11 = w * fz * fy;
  atomicAdd(m + c.r00 + c.x0, w00 * gx);
  atomicAdd(m + c.r00 + c.x1, w00 * fx);
  atomicAdd(m + c.r01 + c.x0, w01 * gx);
  atomicAdd(m + c.r01 + c.x1, w01 * fx);
  atomicAdd(m + c.r10 + c.x0, w10 * gx);
  atomicAdd(m + c.r10 + c.x1, w10 * fx);
  atomicAdd(m + c.r11 + c.x0, w11 * gx);
  atomicAdd(m + c.r11 + c.x1, w11 * fx);
}

}  // namespace
}  // namespace pmlens
