// Warp-level replica culling for the lightcone projection and its transpose.
//
// The particle state is kept sorted by coarse spatial bucket, so the 32
// consecutive particles of a warp occupy a small box of the simulation volume.
// Lane q tests that box, mapped through replica q's rotation / flip / periodic
// shift / offset, against the shell's distance range, the line-of-sight
// half-space and the field of view widened by the displacement margin; a
// ballot gives the replicas any particle of the warp can reach.  The test is
// conservative (the box is widened by a small slack against rounding, and a box
// that straddles the periodic boundary after the transform becomes the whole
// axis), so culled (particle, replica) pairs are exactly pairs the per-particle
// tests would reject: the projection is unchanged, only the work shrinks.
#pragma once

#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pmlens {
namespace {

// Positions in cells (original frame) of the warp's valid lanes lie in
// [lo[a], hi[a]] per axis a.
struct WarpBox {
  float lo[3], hi[3];
};

__device__ __forceinline__ WarpBox warp_box(bool valid, float p0, float p1, float p2) {
  WarpBox b;
  const float inf = __int_as_float(0x7f800000);
  b.lo[0] = valid ? p0 : inf; b.hi[0] = valid ? p0 : -inf;
  b.lo[1] = valid ? p1 : inf; b.hi[1] = valid ? p1 : -inf;
  b.lo[2] = valid ? p2 : inf; b.hi[2] = valid ? p2 : -inf;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = fminf(b.lo[a], __shfl_xor_sync(0xffffffffu, b.lo[a], o));
      b.hi[a] = fmaxf(b.hi[a], __shfl_xor_sync(0xffffffffu, b.hi[a], o));
    }
  }
  return b;
}

// Shell membership, chi^2 in (lo2, hi2], of the replica position (gi + f) cells
// (gi: integer cell including the replica offset, f: fraction).  In FP32 a
// position thousands of cells from the observer carries a rounding of ~1e-7 of
// its distance, which near a shell boundary decides membership differently from
// exact arithmetic (and the affected particle's whole weight moves between
// shells); within 1e-6 (relative, in chi^2) of either boundary the test is
// redone in FP64, so that both precisions select the same particles.  The
// forward, reverse and tangent projections share this test.
// lo2r, hi2r: the bounds rounded to R on the host (no FP64 conversion per test).
template <typename R>
__device__ __forceinline__ bool in_shell(R chi2, const int (&gi)[3], const R (&f)[3], double cell_len, double lo2,
                                         double hi2, R lo2r, R hi2r) {
  if constexpr (sizeof(R) == 8) {
    return chi2 > lo2 && chi2 <= hi2;
  } else {
    const float band = 1e-6f * chi2;
    if (fabsf(chi2 - lo2r) > band && fabsf(chi2 - hi2r) > band) return chi2 > lo2r && chi2 <= hi2r;
    double c2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double x = ((double)gi[d] + (double)f[d]) * cell_len;
      c2 += x * x;
    }
    return c2 > lo2 && c2 <= hi2;
  }
}

// The exact FP64 value of an FP32 number, assembled from its IEEE-754 fields
// with integer operations (normal numbers: exponent rebiased by 1023 - 127,
// mantissa moved to the top of the 52-bit field); zeros, subnormals, infinities
// and NaNs take the conversion instruction.
__device__ __forceinline__ double exact_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)x;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double to_f64(float x) { return exact_f64(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// false only if no position in the box can pass the shell, z > 0 and field-of-view
// tests of the per-particle code under replica rp
__device__ __forceinline__ bool replica_may_hit(const Replica& rp, const WarpBox& b, int M, float cell_len,
                                                float lo2, float hi2, float tan_half, float margin) {
  const float slack = 0.01f;  // cells: covers FP32 rounding of the per-particle positions
  const float Mf = (float)M;
  float bl[3], bh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ax = rp.perm[d];
    float a = ax == 0 ? b.lo[0] : (ax == 1 ? b.lo[1] : b.lo[2]);
    float h = ax == 0 ? b.hi[0] : (ax == 1 ? b.hi[1] : b.hi[2]);
    bool full = !(a <= h);  // empty box (no valid lane): keep it simple, test the whole axis
    if (rp.flip >> d & 1) {
      // p -> M - p for p > 0, and 0 -> 0
      if (a <= 0.f) full = true;
      else { const float na = Mf - h, nh = Mf - a; a = na; h = nh; }
    }
    a += (float)rp.shift[d];
    h += (float)rp.shift[d];
    if (a >= Mf) { a -= Mf; h -= Mf; }
    if (h >= Mf) full = true;  // straddles the periodic boundary
    if (full) { a = 0.f; h = Mf; }
    const float off = (float)rp.n[d] * Mf;
    bl[d] = (a + off - slack) * cell_len;
    bh[d] = (h + off + slack) * cell_len;
  }
  float dmin2 = 0.f, dmax2 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float nearest = bl[d] > 0.f ? bl[d] : (bh[d] < 0.f ? -bh[d] : 0.f);
    const float far = fmaxf(fabsf(bl[d]), fabsf(bh[d]));
    dmin2 += nearest * nearest;
    dmax2 += far * far;
  }
  if (dmax2 <= lo2 || dmin2 > hi2) return false;
  if (bh[2] <= 0.f) return false;
  const float lim = bh[2] * tan_half + margin;
  const float nx = bl[0] > 0.f ? bl[0] : (bh[0] < 0.f ? -bh[0] : 0.f);
  const float ny = bl[1] > 0.f ? bl[1] : (bh[1] < 0.f ? -bh[1] : 0.f);
  return nx <= lim && ny <= lim;
}

// Bit i of the result: replica base + i may be hit by the warp (nrep - base <= 32 used).
__device__ __forceinline__ unsigned cull_replicas(const Replica* rep, int nrep, int base, const WarpBox& b, int M,
                                                  float cell_len, float lo2, float hi2, float tan_half, float margin) {
  const int q = base + (threadIdx.x & 31);
  const bool hit = q < nrep && replica_may_hit(rep[q], b, M, cell_len, lo2, hi2, tan_half, margin);
  return __ballot_sync(0xffffffffu, hit);
}

}  // namespace
}  // namespace pmlens
