// Shared-memory Stockham FFT kernels for the 3D real-to-complex transforms of
// the particle-mesh solver (force mesh and initial-condition lattice).
//
// Data layout: real meshes [z][y][x] (x fastest, no padding); complex
// half-spectra [z][y][P] with P >= n/2 + 1 (row pitch rounded for alignment),
// kx in 0..n/2, ky, kz in 0..n-1 (negative frequencies above n/2).
//
// Passes (all HBM-streaming, one read + one write of the mesh each):
//  * x pass: each row of n reals is packed into n/2 complex values, FFT'd in
//    shared memory and untangled into the n/2+1 half-spectrum (and back);
//  * y / z passes: tiles of W adjacent kx columns (W*8 contiguous bytes per
//    row, full 32-byte sectors) spanning the whole axis, FFT'd along the
//    column in shared memory, written back in place;
//  * the z pass of a force evaluation is fused with the Fourier-space
//    operator: forward z FFT, multiply by each output's kernel (Poisson +
//    gradient, PGD filter, LPT operators), inverse z FFT, store -- the
//    spectrum itself never goes back to HBM.
//
// The 1D transform is a mixed-radix (16, 8, 4, 2, 3) Stockham auto-sort FFT:
// each stage reads the r inputs of a butterfly at stride n/r, applies twiddles
// W_{Ns r}^{(j mod Ns) k} (from a stage-major table, so that the consecutive
// butterflies of a warp read consecutive entries), a radix-r DFT in registers,
// and writes to (j div Ns) Ns r + (j mod Ns) + k Ns, leaving the output in
// natural order.
#pragma once

#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pmlens {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i (forward transforms) or +i (inverse transforms)
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* v) {
  const C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = mul_mi<INV>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* v) {
  using R = decltype(C{}.x);
  const R s = R(0.70710678118654752440);
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o1 *= W8, o2 *= W8^2, o3 *= W8^3 with W8 = exp(-/+ i pi / 4)
  if (!INV) {
    o1 = C{(o1.x + o1.y) * s, (o1.y - o1.x) * s};
    o3 = C{(o3.y - o3.x) * s, -(o3.x + o3.y) * s};
  } else {
    o1 = C{(o1.x - o1.y) * s, (o1.x + o1.y) * s};
    o3 = C{-(o3.x + o3.y) * s, (o3.x - o3.y) * s};
  }
  o2 = mul_mi<INV>(o2);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C* v) {
  using R = decltype(C{}.x);
  const R h = R(0.86602540378443864676);  // sqrt(3)/2
  const C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
  const C m = C{v[0].x - R(0.5) * s.x, v[0].y - R(0.5) * s.y};
  const C t = C{h * d.x, h * d.y};
  v[0] = cadd(v[0], s);
  if (!INV) {
    v[1] = C{m.x + t.y, m.y - t.x};  // m - i t
    v[2] = C{m.x - t.y, m.y + t.x};  // m + i t
  } else {
    v[1] = C{m.x - t.y, m.y + t.x};
    v[2] = C{m.x + t.y, m.y - t.x};
  }
}

// 16 = 4 x 4: X[k1 + 4 k2] = sum_n1 W4^{n1 k2} W16^{n1 k1} sum_n2 W4^{n2 k1} x[n1 + 4 n2]
template <bool INV, typename C> __device__ __forceinline__ void dft16(C* v) {
  using R = decltype(C{}.x);
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);  // cos, sin pi/8
  const R h = R(0.70710678118654752440);
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4<INV>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
  // W16^m, m = n1 k1, for the forward sign; the inverse takes the conjugate
  auto tw = [&](C& a, R wr, R wi) { a = cmul(a, C{wr, INV ? -wi : wi}); };
  tw(v[5], c1, -s1);   // m = 1
  tw(v[6], h, -h);     // m = 2
  tw(v[7], s1, -c1);   // m = 3
  tw(v[9], h, -h);     // m = 2
  v[10] = mul_mi<INV>(v[10]);  // m = 4
  tw(v[11], -h, -h);   // m = 6
  tw(v[13], s1, -c1);  // m = 3
  tw(v[14], -h, -h);   // m = 6
  tw(v[15], -c1, s1);  // m = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose to natural order
  C o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = o[k];
}

template <int RAD, bool INV, typename C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (RAD == 2) dft2<INV>(v);
  else if constexpr (RAD == 3) dft3<INV>(v);
  else if constexpr (RAD == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (RAD == 8) dft8<INV>(v);
  else dft16<INV>(v);
}

template <int... Rs> struct Radices {};
template <int N> struct Plan;
template <> struct Plan<16> { static constexpr int V = 8; using Rad = Radices<8, 2>; };
template <> struct Plan<32> { static constexpr int V = 8; using Rad = Radices<8, 4>; };
template <> struct Plan<48> { static constexpr int V = 24; using Rad = Radices<8, 2, 3>; };
template <> struct Plan<64> { static constexpr int V = 8; using Rad = Radices<8, 8>; };
template <> struct Plan<96> { static constexpr int V = 24; using Rad = Radices<8, 4, 3>; };
template <> struct Plan<128> { static constexpr int V = 8; using Rad = Radices<8, 8, 2>; };
template <> struct Plan<192> { static constexpr int V = 24; using Rad = Radices<8, 8, 3>; };
template <> struct Plan<256> { static constexpr int V = 8; using Rad = Radices<8, 8, 4>; };
template <> struct Plan<512> { static constexpr int V = 8; using Rad = Radices<8, 8, 8>; };
template <> struct Plan<1024> { static constexpr int V = 8; using Rad = Radices<8, 8, 8, 2>; };

// Row FFTs of the x pass: 256 points in two radix-16 stages, one shared-memory
// pass fewer than 8 x 8 x 4 and no stage whose stores fall 2-way on a bank
template <int H> struct RowPlan : Plan<H> {};
template <> struct RowPlan<256> { static constexpr int V = 16; using Rad = Radices<16, 16>; };

// Element k of a unit-stride column sits at pad(k) = k + k / 16: the first
// Stockham stage writes 8 consecutive outputs per thread (stride 8 across
// lanes), which without the pad is a 16-way shared-memory bank conflict.
__device__ __forceinline__ int pad16(int k) { return k + (k >> 4); }
template <int H> struct PadLen { static constexpr int value = H + H / 16; };

// One Stockham stage over CP adjacent columns of N elements at
// buf[row * RS + col * CS] (RS == 1: buf[pad16(row) + col * CS]); T = N / V
// threads per column group, thread t handles V / RAD butterflies of each of
// its CP columns with one set of twiddles.  Two adjacent FP32 columns
// (CS == 1) move as one 16-byte shared-memory access.
// Padded offset pad16(base + k * S) - pad16(base) when it is the same for every
// base of the access pattern: (a) S a multiple of 16; (b) S | 16 and the base
// is a multiple of 16 plus a remainder below S (block writes of a stage with
// Ns * R a multiple of 16); (c) the R outputs of a butterfly sit inside one
// aligned group of 16 (Ns * R | 16).  -1: no constant offset.
template <int S, int R, bool WRITE, int NSR>
__device__ __forceinline__ constexpr int pad_step(int k) {
  if constexpr (S % 16 == 0) return k * S + k * S / 16;
  else if constexpr (WRITE && 16 % S == 0 && NSR % 16 == 0) return k * S + (k * S) / 16;
  else if constexpr (WRITE && 16 % NSR == 0) return k * S;
  else return -1;
}

// Identity load operator of a Stockham stage.
struct NoOp {
  template <typename C> __device__ __forceinline__ C operator()(int, int, C v) const { return v; }
};

// One Stockham stage over CP adjacent columns of N elements at
// buf[row * RS + col * CS] (RS == 1: buf[pad16(row) + col * CS]); T = N / V
// threads per column group, thread t handles V / RAD butterflies of each of
// its CP columns with one set of twiddles.  Two adjacent FP32 columns
// (CS == 1) move as one 16-byte shared-memory access.  The stage reads from
// `src` (which may be `buf`), each element through op(row, column, value) --
// the first stage of a transform applies an elementwise spectral operator as
// it reads, instead of a separate pass over the tile -- and writes to `buf`.
template <typename C, int N, int V, int RAD, bool INV, int NS, int RS, int CS, int CP, typename Op = NoOp>
__device__ __forceinline__ void stage(const C* src, C* buf, int col, int t, const C* tw, const Op& op = Op{}) {
  constexpr bool VEC = CP == 2 && CS == 1 && RS != 1 && sizeof(C) == 8;
  auto at = [&](int row, int cc) -> C& {
    return RS == 1 ? buf[pad16(row) + (col + cc) * CS] : buf[row * RS + (col + cc) * CS];
  };
  auto at_src = [&](int row, int cc) -> const C& {
    return RS == 1 ? src[pad16(row) + (col + cc) * CS] : src[row * RS + (col + cc) * CS];
  };
  constexpr int T = N / V;
  constexpr int NB = V / RAD;
  constexpr int NR = N / RAD;
  // unit-stride (padded) columns: constant offsets from one padded base per butterfly
  constexpr bool RD_CONST = RS == 1 && pad_step<NR, RAD, false, NS * RAD>(1) >= 0;
  constexpr bool WR_CONST = RS == 1 && pad_step<NS, RAD, true, NS * RAD>(1) >= 0;
  C v[CP][NB][RAD];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + b * T;
    if constexpr (RD_CONST && CP == 1) {
      const C* rb = src + pad16(j) + col * CS;
#pragma unroll
      for (int k = 0; k < RAD; ++k) v[0][b][k] = op(j + k * NR, col, rb[pad_step<NR, RAD, false, NS * RAD>(k)]);
    } else {
#pragma unroll
      for (int k = 0; k < RAD; ++k) {
        if constexpr (VEC) {
          const float4 q = *reinterpret_cast<const float4*>(&at_src(j + k * NR, 0));
          v[0][b][k] = op(j + k * NR, col, C{q.x, q.y});
          v[CP - 1][b][k] = op(j + k * NR, col + CP - 1, C{q.z, q.w});
        } else {
#pragma unroll
          for (int cc = 0; cc < CP; ++cc) v[cc][b][k] = op(j + k * NR, col + cc, at_src(j + k * NR, cc));
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + b * T;
    const int jm = j % NS;
    if (NS > 1) {
#pragma unroll
      for (int k = 1; k < RAD; ++k) {
        C w = tw[(k - 1) * NS + jm];
        if (INV) w.y = -w.y;
#pragma unroll
        for (int cc = 0; cc < CP; ++cc) v[cc][b][k] = cmul(v[cc][b][k], w);
      }
    }
#pragma unroll
    for (int cc = 0; cc < CP; ++cc) dft<RAD, INV>(v[cc][b]);
    const int base = (j - jm) * RAD + jm;
    if constexpr (WR_CONST && CP == 1) {
      C* wb = buf + pad16(base) + col * CS;
#pragma unroll
      for (int k = 0; k < RAD; ++k) wb[pad_step<NS, RAD, true, NS * RAD>(k)] = v[0][b][k];
    } else {
      // first stage on 64-byte rows (8 FP32 columns): the lanes of consecutive t write rows
      // RAD t + k, all on the same half of the banks; odd t write the butterfly's outputs in
      // pair-swapped order (row k ^ 1), so that each store instruction covers every bank
      constexpr bool SWAP = NS == 1 && RS != 1 && RS * (int)sizeof(C) == 64 && RAD % 2 == 0;
      const int sw = SWAP ? (t & 1) : 0;
#pragma unroll
      for (int k = 0; k < RAD; ++k) {
        const int kk = k ^ sw;
        if constexpr (VEC) {
          const C a = SWAP && sw ? v[0][b][k ^ 1] : v[0][b][k];
          const C c = SWAP && sw ? v[CP - 1][b][k ^ 1] : v[CP - 1][b][k];
          *reinterpret_cast<float4*>(&at(base + kk * NS, 0)) = make_float4(a.x, a.y, c.x, c.y);
        } else {
#pragma unroll
          for (int cc = 0; cc < CP; ++cc) at(base + kk * NS, cc) = SWAP && sw ? v[cc][b][k ^ 1] : v[cc][b][k];
        }
      }
    }
  }
  __syncthreads();
}

template <typename C, int N, int V, bool INV, int RS, int CS, int CP, int NS, typename Op, int RAD, int... Rest>
__device__ __forceinline__ void run_stages(const C* src, C* buf, int col, int t, const C* tw, const Op& op) {
  stage<C, N, V, RAD, INV, NS, RS, CS, CP, Op>(src, buf, col, t, tw, op);
  if constexpr (sizeof...(Rest) > 0)
    run_stages<C, N, V, INV, RS, CS, CP, NS * RAD, NoOp, Rest...>(buf, buf, col, t, NS > 1 ? tw + (RAD - 1) * NS : tw,
                                                                  NoOp{});
}

template <typename C, int N, int V, bool INV, int RS, int CS, int CP, typename Op, int... Rs>
__device__ __forceinline__ void fft_column_impl(Radices<Rs...>, const C* src, C* buf, int col, int t, const C* tw,
                                                const Op& op) {
  run_stages<C, N, V, INV, RS, CS, CP, 1, Op, Rs...>(src, buf, col, t, tw, op);
}

// In-place FFT of CP adjacent columns of length N held in shared memory:
// element k of column `col + c` at buf[k * RS + (col + c) * CS] (compile-time
// strides), with the radices and elements per thread of plan PL.
template <typename C, int N, bool INV, int RS, int CS, int CP = 1, typename PL = Plan<N>>
__device__ __forceinline__ void fft_column(C* buf, int col, int t, const C* tw) {
  fft_column_impl<C, N, PL::V, INV, RS, CS, CP, NoOp>(typename PL::Rad{}, buf, buf, col, t, tw, NoOp{});
}

// The same transform of op(row, column, src element) into buf (src may be buf): an
// elementwise spectral operator applied as the first stage reads.
template <typename C, int N, bool INV, int RS, int CS, int CP = 1, typename PL = Plan<N>, typename Op>
__device__ __forceinline__ void fft_column_from(const C* src, C* buf, int col, int t, const C* tw, const Op& op) {
  fft_column_impl<C, N, PL::V, INV, RS, CS, CP, Op>(typename PL::Rad{}, src, buf, col, t, tw, op);
}

// Stage-major twiddles of the plan of N: for each stage with NS > 1, in order,
// the block tw[(k - 1) * NS + jm] = exp(-2 pi i jm k / (NS RAD)), k = 1..RAD-1,
// jm < NS.  Threads that hold consecutive butterflies (consecutive jm) read
// consecutive entries; in a table indexed by jm k N / (NS RAD) their reads
// fell at strides that share banks.  N - RAD_1 entries in all (fewer than N).
template <typename C, int NS, int RAD, int... Rest>
__device__ __forceinline__ void fill_stage_twiddles(C* tw) {
  using R = decltype(C{}.x);
  if constexpr (NS > 1) {
    for (int m = threadIdx.x; m < (RAD - 1) * NS; m += blockDim.x) {
      const int k = m / NS + 1, jm = m - (k - 1) * NS;
      R s, c;
      if constexpr (sizeof(R) == 4) sincospif(-2.0f * (float)(jm * k) / (float)(NS * RAD), &s, &c);
      else sincospi(-2.0 * (double)(jm * k) / (double)(NS * RAD), &s, &c);
      tw[m] = C{c, s};
    }
  }
  if constexpr (sizeof...(Rest) > 0) fill_stage_twiddles<C, NS * RAD, Rest...>(NS > 1 ? tw + (RAD - 1) * NS : tw);
}

template <typename C, int... Rs>
__device__ __forceinline__ void fill_plan_twiddles(Radices<Rs...>, C* tw) {
  fill_stage_twiddles<C, 1, Rs...>(tw);
}

template <typename C, int N, typename PL = Plan<N>> __device__ __forceinline__ void make_twiddles(C* tw) {
  fill_plan_twiddles<C>(typename PL::Rad{}, tw);
}

// tu[k] = exp(-2 pi i k / N), k <= N / 2 (real <-> half-length complex untangling)
template <typename C, int N> __device__ __forceinline__ void make_untangle(C* tu) {
  using R = decltype(C{}.x);
  for (int m = threadIdx.x; m <= N / 2; m += blockDim.x) {
    R s, c;
    if constexpr (sizeof(R) == 4) sincospif(-2.0f * (float)m / (float)N, &s, &c);
    else sincospi(-2.0 * (double)m / (double)N, &s, &c);
    tu[m] = C{c, s};
  }
}

// ------------------------------------------------------------ tile widths
// CP: columns per thread (two adjacent FP32 columns share twiddles, index
// arithmetic and 16-byte shared-memory accesses)
template <typename R, int N> struct ColTile {
  static constexpr int cap_smem = (sizeof(R) == 4 ? 8192 : 4096) / N;  // N*W*sizeof(C) <= 64 KB
  static constexpr int cap_thr = 1024 * Plan<N>::V / N;
  static constexpr int cap = cap_smem < cap_thr ? (cap_smem < 32 ? cap_smem : 32) : (cap_thr < 32 ? cap_thr : 32);
  static constexpr int W = cap >= 32 ? 32 : cap >= 16 ? 16 : cap >= 8 ? 8 : cap >= 4 ? 4 : cap >= 2 ? 2 : 1;
  static constexpr int CP = (sizeof(R) == 4 && W >= 2) ? 2 : 1;
  static constexpr int THREADS = W / CP * (N / Plan<N>::V);
};

// fused z pass: half the column tile of the plain passes for large N, so that
// several blocks (A/B buffer pairs) share an SM and overlap load and compute
template <typename R, int N> struct ZTile {
  static constexpr int W = (N >= 256 && ColTile<R, N>::W >= 4) ? ColTile<R, N>::W / 2 : ColTile<R, N>::W;
  static constexpr int CP = (sizeof(R) == 4 && W >= 2) ? 2 : 1;
  static constexpr int THREADS = W / CP * (N / Plan<N>::V);
  static constexpr int SMEM = (N + 2 * N * W) * (int)sizeof(R) * 2;
  // two resident blocks: the operator passes need ~128 registers per thread
  // (a third block's register cap spills, measured slower)
  static constexpr int MINB = (227 * 1024 / SMEM) >= 2 ? 2 : 1;
};

template <typename R, int N> struct RowTile {  // x pass: rows of N reals, FFT length N/2
  static constexpr int H = N / 2;
  using PL = RowPlan<H>;
  static constexpr int T = H / PL::V;
  static constexpr int ROWS = (256 / T) > 0 ? (256 / T) : 1;
  static constexpr int THREADS = ROWS * T;
  // twiddles, untangle table and the padded rows
  static constexpr int SMEM = (H + H + 2 + ROWS * (PadLen<H>::value + 1)) * 2 * (int)sizeof(R);
};

// ------------------------------------------------------------ tile copies
// Copy a W-column x N-row tile between global memory (row stride rstride,
// columns >= nv absent) and shared memory [row][W].  Every thread issues all
// of its loads before the first shared-memory store, so that each SM keeps
// enough bytes in flight to cover the HBM latency; FP32 tiles move as
// 16-byte pairs of complex values.
template <typename R, int N, int W, int THREADS>
__device__ __forceinline__ void load_tile(typename CT<R>::T* dst, const typename CT<R>::T* src, long long rstride,
                                          int nv) {
  using C = typename CT<R>::T;
  if constexpr (sizeof(R) == 4 && W % 2 == 0) {
    constexpr int WP = W / 2, PER = N * WP / THREADS;
    static_assert(N * WP % THREADS == 0, "tile split");
    float4 v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / WP, c = 2 * (e - row * WP);
      const C* g = src + row * rstride + c;
      if (c + 1 < nv) v[q] = *reinterpret_cast<const float4*>(g);
      else if (c < nv) { const C a = g[0]; v[q] = make_float4(a.x, a.y, 0.f, 0.f); }
      else v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) reinterpret_cast<float4*>(dst)[threadIdx.x + q * THREADS] = v[q];
  } else {
    constexpr int PER = N * W / THREADS;
    static_assert(N * W % THREADS == 0, "tile split");
    C v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / W, c = e - row * W;
      v[q] = c < nv ? src[row * rstride + c] : C{0, 0};
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) dst[threadIdx.x + q * THREADS] = v[q];
  }
}

template <typename R, int N, int W, int THREADS>
__device__ __forceinline__ void store_tile(typename CT<R>::T* dst, const typename CT<R>::T* src, long long rstride,
                                           int nv) {
  using C = typename CT<R>::T;
  if constexpr (sizeof(R) == 4 && W % 2 == 0) {
    constexpr int WP = W / 2, PER = N * WP / THREADS;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / WP, c = 2 * (e - row * WP);
      const float4 v = reinterpret_cast<const float4*>(src)[e];
      C* g = dst + row * rstride + c;
      if (c + 1 < nv) *reinterpret_cast<float4*>(g) = v;
      else if (c < nv) g[0] = C{v.x, v.y};
    }
  } else {
    constexpr int PER = N * W / THREADS;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / W, c = e - row * W;
      if (c < nv) dst[row * rstride + c] = src[e];
    }
  }
}

// store i k * tile: k = k_x of each column (per_column) or the scalar `kc`
template <typename R, int N, int W, int THREADS>
__device__ __forceinline__ void store_tile_ik(typename CT<R>::T* dst, const typename CT<R>::T* src, long long rstride,
                                              int nv, int kx0, R kf, R kc, bool per_column) {
  using C = typename CT<R>::T;
  constexpr int h = N / 2;
  auto kof = [&](int c) -> R {
    const int ix = kx0 + c;
    return per_column ? (ix == h ? R(0) : kf * (R)(ix <= h ? ix : ix - N)) : kc;
  };
  if constexpr (sizeof(R) == 4 && W % 2 == 0) {
    constexpr int WP = W / 2, PER = N * WP / THREADS;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / WP, c = 2 * (e - row * WP);
      const float4 v = reinterpret_cast<const float4*>(src)[e];
      const R k0 = kof(c), k1 = kof(c + 1);
      const float4 o = make_float4(-k0 * v.y, k0 * v.x, -k1 * v.w, k1 * v.z);
      C* g = dst + row * rstride + c;
      if (c + 1 < nv) *reinterpret_cast<float4*>(g) = o;
      else if (c < nv) g[0] = C{o.x, o.y};
    }
  } else {
    constexpr int PER = N * W / THREADS;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * THREADS;
      const int row = e / W, c = e - row * W;
      const R k = kof(c);
      const C b = src[e];
      if (c < nv) dst[row * rstride + c] = C{-k * b.y, k * b.x};
    }
  }
}

// ---------------------------------------------------------------- kernels
// x pass, forward: real rows -> half-spectrum rows
template <typename R, int N>
__global__ void __launch_bounds__(RowTile<R, N>::THREADS)
k_fft_x_r2c(const R* __restrict__ in, typename CT<R>::T* __restrict__ out, int P) {
  using C = typename CT<R>::T;
  constexpr int H = N / 2, ROWS = RowTile<R, N>::ROWS, T = RowTile<R, N>::T, LD = PadLen<H>::value + 1;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* tu = tw + H;        // untangle twiddles exp(-2 pi i k / N), k <= H
  C* buf = tu + H + 2;
  make_twiddles<C, H, typename RowTile<R, N>::PL>(tw);
  make_untangle<C, N>(tu);
  const long long row0 = (long long)blockIdx.x * ROWS;
  {
    // ROWS consecutive rows are contiguous: ROWS * H complex values, read as pairs
    constexpr int THR = RowTile<R, N>::THREADS;
    const C* inc = reinterpret_cast<const C*>(in) + row0 * H;
    if constexpr (sizeof(R) == 4) {
      constexpr int PER = ROWS * H / 2 / THR;
      float4 v[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) v[q] = reinterpret_cast<const float4*>(inc)[threadIdx.x + q * THR];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = 2 * (threadIdx.x + q * THR);
        const int h = e / H, m = e - h * H;
        buf[h * LD + pad16(m)] = C{v[q].x, v[q].y};
        buf[h * LD + pad16(m + 1)] = C{v[q].z, v[q].w};
      }
    } else {
      constexpr int PER = ROWS * H / THR;
      C v[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) v[q] = inc[threadIdx.x + q * THR];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * THR;
        const int h = e / H, m = e - h * H;
        buf[h * LD + pad16(m)] = v[q];
      }
    }
  }
  __syncthreads();
  const int h = threadIdx.x / T, t = threadIdx.x - h * T;
  fft_column<C, H, false, 1, LD, 1, typename RowTile<R, N>::PL>(buf, h, t, tw);
  // X[k] = (Z[k] + conj Z[H-k]) / 2 + e^{-2 pi i k / N} (Z[k] - conj Z[H-k]) / (2i), k <= H
  C* outb = out + row0 * P;
  auto untangle = [&](int hh, int k) {
    const C zk = buf[hh * LD + pad16(k % H)];
    const C zm = cconj(buf[hh * LD + pad16((H - k) % H)]);
    const C ev = C{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y + zm.y)};
    const C od = C{R(0.5) * (zk.y - zm.y), -R(0.5) * (zk.x - zm.x)};  // (zk - zm) / (2i)
    outb[hh * P + k] = cadd(ev, cmul(tu[k], od));
  };
  for (int e = threadIdx.x; e < ROWS * H; e += blockDim.x) {
    const int hh = e / H;
    untangle(hh, e - hh * H);
  }
  for (int hh = threadIdx.x; hh < ROWS; hh += blockDim.x) untangle(hh, H);
}

// x pass, forward, of FP32 meshes stored interleaved per cell (the adjoint's cotangent
// meshes, painted with one vector reduction per corner): rows of N cells -> one
// half-spectrum row per component.  The component rows of a block share the
// shared-memory stages of one x r2c.  A quarter of the x pass's rows per block (4 row
// triples at N = 512: 30 KB of shared memory, 64 threads): more resident blocks hide the
// vector loads (measured 4 ms per pm256 reverse sweep faster than 16 or 8 row triples).
template <int N, int NL> struct RowTileIL {
  static constexpr int H = N / 2, T = RowTile<float, N>::T, LD = PadLen<H>::value + 1;
  static constexpr int ROWS = RowTile<float, N>::ROWS / 4 > 0 ? RowTile<float, N>::ROWS / 4 : 1;
  static constexpr int THREADS = ROWS * T;
  static constexpr int SMEM = (H + H + 2 + NL * ROWS * LD) * 8;
};

struct ILOut { float2* p[4]; };

template <int LANES> struct LaneVec;
template <> struct LaneVec<4> {
  using T = float4;
  __device__ static float get(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
};
template <> struct LaneVec<2> {
  using T = float2;
  __device__ static float get(const float2& v, int c) { return c == 0 ? v.x : v.y; }
};

// x pass of a mesh interleaved per cell (LANES = 4: float4, LANES = 2: float2):
// the first NL lanes of each row are transformed as NL real rows into NL half
// spectra (out.p[0 .. NL-1]).
template <int N, int LANES, int NL>
__global__ void __launch_bounds__(RowTileIL<N, NL>::THREADS)
k_fft_x_r2c_il(const float* __restrict__ in_f, ILOut out, int P) {
  using C = float2;
  using VT = typename LaneVec<LANES>::T;
  constexpr int H = N / 2, ROWS = RowTileIL<N, NL>::ROWS, T = RowTileIL<N, NL>::T, LD = RowTileIL<N, NL>::LD;
  constexpr int THR = RowTileIL<N, NL>::THREADS;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* tu = tw + H;
  C* buf = tu + H + 2;  // component q's rows at buf + q * ROWS * LD
  make_twiddles<C, H, typename RowTile<float, N>::PL>(tw);
  make_untangle<C, N>(tu);
  const long long row0 = (long long)blockIdx.x * ROWS;
  {
    // cells 2m and 2m + 1 of a row make complex element m of each component's half-length row
    const VT* inr = reinterpret_cast<const VT*>(in_f) + row0 * N;
    constexpr int PER = ROWS * H / THR, B = PER < 4 ? PER : 4;
    static_assert(PER % B == 0, "load batches");
#pragma unroll 1
    for (int q0 = 0; q0 < PER; q0 += B) {
      VT a[B], b[B];
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int e = threadIdx.x + (q0 + q) * THR;
        a[q] = inr[2 * e];
        b[q] = inr[2 * e + 1];
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int e = threadIdx.x + (q0 + q) * THR;
        const int hh = e / H, m = e - hh * H;
        const int o = hh * LD + pad16(m);
#pragma unroll
        for (int c = 0; c < NL; ++c) buf[c * ROWS * LD + o] = C{LaneVec<LANES>::get(a[q], c), LaneVec<LANES>::get(b[q], c)};
      }
    }
  }
  __syncthreads();
  const int h = threadIdx.x / T, t = threadIdx.x - h * T;
#pragma unroll 1
  for (int q = 0; q < NL; ++q) fft_column<C, H, false, 1, LD, 1, typename RowTile<float, N>::PL>(buf + q * ROWS * LD, h, t, tw);
  // X[k] = (Z[k] + conj Z[H-k]) / 2 + e^{-2 pi i k / N} (Z[k] - conj Z[H-k]) / (2i), k <= H
#pragma unroll 1
  for (int q = 0; q < NL; ++q) {
    const C* bq = buf + q * ROWS * LD;
    float2* outb = out.p[q] + row0 * P;
    auto untangle = [&](int hh, int k) {
      const C zk = bq[hh * LD + pad16(k % H)];
      const C zm = cconj(bq[hh * LD + pad16((H - k) % H)]);
      const C ev = C{0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y)};
      const C od = C{0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x)};
      outb[hh * P + k] = cadd(ev, cmul(tu[k], od));
    };
    for (int e = threadIdx.x; e < ROWS * H; e += blockDim.x) {
      const int hh = e / H;
      untangle(hh, e - hh * H);
    }
    for (int hh = threadIdx.x; hh < ROWS; hh += blockDim.x) untangle(hh, H);
  }
}

// x pass, inverse: half-spectrum rows -> real rows (unnormalised: n * IDFT).
// Persistent over blocks of ROWS rows: with pair loads, the next block's input is
// requested right after the current one has been untangled into shared memory,
// so that its HBM latency overlaps the shared-memory FFT.
template <typename R, int N>
__global__ void __launch_bounds__(RowTile<R, N>::THREADS)
k_fft_x_c2r(const typename CT<R>::T* __restrict__ in, R* __restrict__ out, int P, int nblk) {
  using C = typename CT<R>::T;
  constexpr int H = N / 2, ROWS = RowTile<R, N>::ROWS, T = RowTile<R, N>::T, LD = PadLen<H>::value + 1;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + H + H + 2;
  make_twiddles<C, H, typename RowTile<R, N>::PL>(tw);
  constexpr int THR = RowTile<R, N>::THREADS;
  // Z[k] = (X[k] + conj X[H-k]) + i w_k (X[k] - conj X[H-k]), w_k = exp(2 pi i k / N)
  auto untangle = [](C a, C b, C w) {
    const C bm = cconj(b);
    const C ev = cadd(a, bm);
    const C od = cmul(w, csub(a, bm));
    return C{ev.x - od.y, ev.y + od.x};  // ev + i od
  };
  auto untwiddle = [](int k) {
    R s, c;
    if constexpr (sizeof(R) == 4) sincospif(2.0f * (float)k / (float)N, &s, &c);
    else sincospi(2.0 * (double)k / (double)N, &s, &c);
    return C{c, s};
  };
  const int h = threadIdx.x / T, t = threadIdx.x - h * T;
  auto transform_store = [&](int blk) {
    __syncthreads();
    fft_column<C, H, true, 1, LD, 1, typename RowTile<R, N>::PL>(buf, h, t, tw);
    C* outc = reinterpret_cast<C*>(out) + (long long)blk * ROWS * H;
    for (int e = threadIdx.x; e < ROWS * H; e += blockDim.x) {
      const int hh = e / H, m = e - hh * H;
      outc[e] = buf[hh * LD + pad16(m)];
    }
    __syncthreads();  // buf is refilled by the next block's untangling
  };
  if constexpr (THR % (H / 2) == 0) {
    // every input read once: the thread of pair k < H/2 reads X[k] and X[H - k] and writes
    // Z[k] and Z[H - k] (w_{H-k} = -conj w_k); the thread of pair 0 also reads X[H/2]
    constexpr int PER = ROWS * (H / 2) / THR;
    const int k = threadIdx.x % (H / 2);
    C xa[PER], xb[PER], xc[PER];
    auto load = [&](int blk) {
      const C* inb = in + (long long)blk * ROWS * P;  // 32-bit offsets within the block's rows
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int hq = (threadIdx.x + q * THR) / (H / 2);
        xa[q] = inb[hq * P + k];
        xb[q] = inb[hq * P + (H - k)];
        if (k == 0) xc[q] = inb[hq * P + H / 2];
      }
    };
    const C w = untwiddle(k), wm = C{-w.x, w.y};
    int blk = blockIdx.x;
    if (blk < nblk) load(blk);
    for (; blk < nblk; blk += gridDim.x) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int hq = (threadIdx.x + q * THR) / (H / 2);
        buf[hq * LD + pad16(k)] = untangle(xa[q], xb[q], w);
        if (k > 0) buf[hq * LD + pad16(H - k)] = untangle(xb[q], xa[q], wm);
        else buf[hq * LD + pad16(H / 2)] = untangle(xc[q], xc[q], C{R(0), R(1)});
      }
      if (blk + (int)gridDim.x < nblk) load(blk + gridDim.x);
      transform_store(blk);
    }
  } else {
    constexpr int PER = ROWS * H / THR;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
      const C* inb = in + (long long)blk * ROWS * P;
      C vk[PER], vm[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * THR;
        const int hq = e / H, k = e - hq * H;
        vk[q] = inb[hq * P + k];
        vm[q] = inb[hq * P + (H - k)];
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * THR;
        const int hq = e / H, k = e - hq * H;
        buf[hq * LD + pad16(k)] = untangle(vk[q], vm[q], untwiddle(k));
      }
      transform_store(blk);
    }
  }
}

// y or z pass in place: column tiles of W kx values over a full axis.
template <typename R, int N, bool INV>
__global__ void __launch_bounds__(ColTile<R, N>::THREADS, (1024 / ColTile<R, N>::THREADS) > 0 ? 1024 / ColTile<R, N>::THREADS : 1)
k_fft_cols(typename CT<R>::T* __restrict__ data, long long plane_stride, long long row_stride, int ncols) {
  using C = typename CT<R>::T;
  constexpr int W = ColTile<R, N>::W;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + N;
  make_twiddles<C, N>(tw);
  const int kx0 = blockIdx.x * W;
  C* base = data + (long long)blockIdx.y * plane_stride + kx0;
  const int nv = min(W, ncols - kx0);
  load_tile<R, N, W, ColTile<R, N>::THREADS>(buf, base, row_stride, nv);
  __syncthreads();
  constexpr int CP = ColTile<R, N>::CP;
  const int col = CP * (threadIdx.x % (W / CP)), t = threadIdx.x / (W / CP);
  fft_column<C, N, INV, W, 1, CP>(buf, col, t, tw);
  store_tile<R, N, W, ColTile<R, N>::THREADS>(base, buf, row_stride, nv);
}

struct OutPtrs { void* p[9]; };

// PGD filter O_L O_S = exp(-(k_l/k)^2) exp(-(k/k_s)^n) (Eq. 12-13) at k^2 > 0, inv = 1/k^2.
// FP32 evaluates it in log space with the hardware exp/log approximations
// ((k/k_s)^n = exp(n (ln k^2 / 2 - ln k_s)); relative error ~1e-6, far below
// the FP32 path's tolerance); FP64 uses the libm functions.
template <typename R>
__device__ __forceinline__ R pgd_filter(const SpecParams& sp, R k2, R inv) {
  if constexpr (sizeof(R) == 4) {
    const float kl2 = (float)(sp.kl * sp.kl), nexp = (float)sp.nexp, lks = __logf((float)sp.ks);
    return __expf(-kl2 * inv - __expf(nexp * (0.5f * __logf(k2) - lks)));
  } else {
    return exp(-(sp.kl * sp.kl) * inv) * exp(-pow(sqrt(k2) / sp.ks, sp.nexp));
  }
}

// Fourier-space operator of output o at integer frequencies: multiplier re + i im.
template <typename R>
__device__ __forceinline__ void spec_coef(const SpecParams& sp, int o, int ix, int iy, int iz, int n, R& re, R& im) {
  const int h = n / 2;
  const int fx = ix <= h ? ix : ix - n, fy = iy <= h ? iy : iy - n, fz = iz <= h ? iz : iz - n;
  const R kf = (R)sp.kf;
  const R kx = kf * fx, ky = kf * fy, kz = kf * fz;
  const R k2 = kx * kx + ky * ky + kz * kz;
  const R inv = k2 > R(0) ? R(1) / k2 : R(0);
  // odd factors vanish on their axis' Nyquist plane
  const R ox = ix == h ? R(0) : kx, oy = iy == h ? R(0) : ky, oz = iz == h ? R(0) : kz;
  re = 0;
  im = 0;
  switch (sp.op) {
    case OP_FORCE:
    case OP_FORCE_PGD: {
      const R odd = o % 3 == 0 ? ox : (o % 3 == 1 ? oy : oz);
      R s = (R)sp.scale;
      if (o >= 3) s = k2 > R(0) ? (R)sp.pgd_scale * pgd_filter<R>(sp, k2, inv) : R(0);
      im = s * odd * inv;
      break;
    }
    case OP_LPT1:
    case OP_LPT2_DERIV: {
      const R amp = (R)sp.sqrtp[fx * fx + fy * fy + fz * fz] * (R)sp.scale;
      if (o < 3) {
        const R odd = o == 0 ? ox : (o == 1 ? oy : oz);
        im = amp * odd * inv;
      } else {
        // Psi1_{i,j} = -k_i k_j / k^2 delta: (0,0),(1,1),(2,2),(0,1),(0,2),(1,2)
        const int q = o - 3;
        R f;
        if (q == 0) f = kx * kx;
        else if (q == 1) f = ky * ky;
        else if (q == 2) f = kz * kz;
        else if (q == 3) f = ox * oy;
        else if (q == 4) f = ox * oz;
        else f = oy * oz;
        re = -amp * f * inv;
      }
      break;
    }
    case OP_GRAD_NEG: {
      const R odd = o == 0 ? ox : (o == 1 ? oy : oz);
      im = -(R)sp.scale * odd * inv;
      break;
    }
    default:
      re = (R)sp.scale;
  }
}

// g(k) of the force (3/2 Om scale / k^2) or PGD (alpha O_L O_S scale / k^2) operators,
// whose j-th output multiplies by i k_j g(k)
template <typename R>
__device__ __forceinline__ R force_g(const SpecParams& sp, bool pgd, int ix, int iy, int iz, int n) {
  const int h = n / 2;
  const int fx = ix <= h ? ix : ix - n, fy = iy <= h ? iy : iy - n, fz = iz <= h ? iz : iz - n;
  const R kf = (R)sp.kf;
  const R k2 = kf * kf * (R)(fx * fx + fy * fy + fz * fz);
  if (!(k2 > R(0))) return R(0);
  const R inv = R(1) / k2;
  if (!pgd) return (R)sp.scale * inv;
  return (R)sp.pgd_scale * inv * pgd_filter<R>(sp, k2, inv);
}

template <typename R>
__device__ __forceinline__ typename CT<R>::T spec_mult(const SpecParams& sp, int o, int ix, int iy, int iz,
                                                       int n, typename CT<R>::T a) {
  using C = typename CT<R>::T;
  R re, im;
  spec_coef<R>(sp, o, ix, iy, iz, n, re, im);
  return C{re * a.x - im * a.y, re * a.y + im * a.x};
}

// fused z pass: forward z FFT, per-output multiplier, inverse z FFT, store.
template <typename R, int N>
__global__ void __launch_bounds__(ZTile<R, N>::THREADS, ZTile<R, N>::MINB)
k_zpass_op(const typename CT<R>::T* __restrict__ in, OutPtrs outs, int nout, int P, SpecParams sp) {
  using C = typename CT<R>::T;
  constexpr int W = ZTile<R, N>::W, CP = ZTile<R, N>::CP;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* A = tw + N;
  C* B = A + N * W;
  make_twiddles<C, N>(tw);
  const int ncols = N / 2 + 1;
  const int kx0 = blockIdx.x * W;
  const int iy = blockIdx.y;
  const long long plane = (long long)iy * P + kx0;
  const long long rstride = (long long)N * P;
  const int nv = min(W, ncols - kx0);
  load_tile<R, N, W, ZTile<R, N>::THREADS>(A, in + plane, rstride, nv);
  __syncthreads();
  const int col = CP * (threadIdx.x % (W / CP)), t = threadIdx.x / (W / CP);
  fft_column<C, N, false, W, 1, CP>(A, col, t, tw);
  constexpr int THR = ZTile<R, N>::THREADS;
  constexpr int EPT = N * W / THR;  // elements per thread, the same set in every loop below
  const bool force = sp.op == OP_FORCE || sp.op == OP_FORCE_PGD;
  if (force) {
    // i k_x and i k_y are constant along a z column: F_x = i k_x IFFT_z(g A) and
    // F_y = i k_y IFFT_z(g A) share one inverse transform; F_z = IFFT_z(i k_z g A)
    // needs its own.  A is scaled in place, first by g = (3/2) Om / k^2, then
    // (PGD outputs) by gp / g = (alpha / (3/2 Om)) O_L O_S, so that no
    // per-element factor is kept in registers; the last transform runs on A.
    const R kf = (R)sp.kf;
    const int h = N / 2;
    const R oy = iy == h ? R(0) : kf * (R)(iy <= h ? iy : iy - N);
    const int fy = iy <= h ? iy : iy - N;
    const int npass = nout == 6 ? 4 : 2;
    const R pratio = (R)(sp.pgd_scale / sp.scale);
    for (int pass = 0; pass < npass; ++pass) {
      const bool zc = pass & 1;  // the z component's transform
      const bool last = pass == npass - 1;
      C* T = last ? A : B;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * THR;
        const int row = e / W, c = e - row * W, ix = kx0 + c;
        C a = A[e];
        if (!zc) {
          const int fx = ix <= h ? ix : ix - N, fz = row <= h ? row : row - N;
          const R k2 = kf * kf * (R)(fx * fx + fy * fy + fz * fz);
          const R inv = k2 > R(0) ? R(1) / k2 : R(0);
          const R f = pass == 0 ? (R)sp.scale * inv : (k2 > R(0) ? pratio * pgd_filter<R>(sp, k2, inv) : R(0));
          a = C{f * a.x, f * a.y};
          A[e] = a;
          T[e] = a;
        } else {
          const R oz = row == h ? R(0) : kf * (R)(row <= h ? row : row - N);
          T[e] = C{-oz * a.y, oz * a.x};  // i k_z a
        }
      }
      __syncthreads();
      fft_column<C, N, true, W, 1, CP>(T, col, t, tw);
      const int o0 = pass >= 2 ? 3 : 0;
      if (zc) {
        store_tile<R, N, W, THR>(reinterpret_cast<C*>(outs.p[o0 + 2]) + plane, T, rstride, nv);
      } else if (sp.err) {
        // G itself: the dual inverse y pass applies i k_x and i k_y
        store_tile<R, N, W, THR>(reinterpret_cast<C*>(outs.p[o0]) + plane, T, rstride, nv);
      } else {
        // two outputs from one transform: i k_x (per column) and i k_y (per block) times it
        store_tile_ik<R, N, W, THR>(reinterpret_cast<C*>(outs.p[o0]) + plane, T, rstride, nv, kx0, kf, R(0), true);
        store_tile_ik<R, N, W, THR>(reinterpret_cast<C*>(outs.p[o0 + 1]) + plane, T, rstride, nv, kx0, kf, oy, false);
      }
      __syncthreads();
    }
  } else {
    for (int o = 0; o < nout; ++o) {
      for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
        const int row = e / W, c = e - row * W;
        B[e] = spec_mult<R>(sp, o, kx0 + c, iy, row, N, A[e]);
      }
      __syncthreads();
      fft_column<C, N, true, W, 1, CP>(B, col, t, tw);
      store_tile<R, N, W, THR>(reinterpret_cast<C*>(outs.p[o]) + plane, B, rstride, nv);
      __syncthreads();
    }
  }
}

struct InPtrs { const void* p[9]; };

// transposed fused z pass: B = sum_c conj(m_{first+c}(k)) FFT_z(A_c); store IFFT_z(B)
template <typename R, int N>
__global__ void __launch_bounds__(ZTile<R, N>::THREADS, ZTile<R, N>::MINB)
k_zpass_combine(InPtrs ins, int nin, int first, typename CT<R>::T* __restrict__ out, int P, SpecParams sp) {
  using C = typename CT<R>::T;
  constexpr int W = ZTile<R, N>::W;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* A = tw + N;
  C* B = A + N * W;
  make_twiddles<C, N>(tw);
  const int ncols = N / 2 + 1;
  const int kx0 = blockIdx.x * W;
  const int iy = blockIdx.y;
  const long long plane = (long long)iy * P + kx0;
  const long long rstride = (long long)N * P;
  const int nv = min(W, ncols - kx0);
  constexpr int CP = ZTile<R, N>::CP;
  const int col = CP * (threadIdx.x % (W / CP)), t = threadIdx.x / (W / CP);
  for (int e = threadIdx.x; e < N * W; e += blockDim.x) B[e] = C{0, 0};
  // force / PGD groups of three (x, y, z components): nin == 3 (one group, first 0 or 3) or
  // nin == 6 with first == 0 (the force group, then the PGD group, at the same positions)
  const bool fop = sp.op == OP_FORCE || sp.op == OP_FORCE_PGD;
  const int ngroups = !fop ? 0 : (nin == 3 && (first == 0 || first == 3)) ? 1 : (nin == 6 && first == 0) ? 2 : 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    // conj(i k_x g) FFT(A_x) + conj(i k_y g) FFT(A_y) = -i g FFT(k_x A_x + k_y A_y):
    // k_x, k_y are constant along the column, so one forward transform serves both
    const int base = 3 * gi, gfirst = first + base;
    constexpr int THR = ZTile<R, N>::THREADS;
    constexpr int EPT = N * W / THR;
    const R kf = (R)sp.kf;
    const int h = N / 2;
    const R oy = iy == h ? R(0) : kf * (R)(iy <= h ? iy : iy - N);
    load_tile<R, N, W, THR>(A, reinterpret_cast<const C*>(ins.p[base]) + plane, rstride, nv);
    __syncthreads();
    {
      const C* iny = reinterpret_cast<const C*>(ins.p[base + 1]) + plane;
      C vy[EPT];
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * THR;
        const int row = e / W, cc = e - row * W;
        vy[q] = cc < nv ? iny[row * rstride + cc] : C{0, 0};
      }
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * THR;
        const int ix = kx0 + (e - (e / W) * W);
        const R ox = ix == h ? R(0) : kf * (R)(ix <= h ? ix : ix - N);
        const C a = A[e];
        A[e] = C{ox * a.x + oy * vy[q].x, ox * a.y + oy * vy[q].y};
      }
    }
    __syncthreads();
    fft_column<C, N, false, W, 1, CP>(A, col, t, tw);
    for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
      const int row = e / W, cc = e - row * W;
      const R g = force_g<R>(sp, gfirst >= 3, kx0 + cc, iy, row, N);
      const C a = A[e];
      B[e] = C{B[e].x + g * a.y, B[e].y - g * a.x};  // + (-i g a)
    }
    __syncthreads();
    load_tile<R, N, W, THR>(A, reinterpret_cast<const C*>(ins.p[base + 2]) + plane, rstride, nv);
    __syncthreads();
    fft_column<C, N, false, W, 1, CP>(A, col, t, tw);
    for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
      const int row = e / W, cc = e - row * W;
      R re, im;
      spec_coef<R>(sp, gfirst + 2, kx0 + cc, iy, row, N, re, im);
      const C a = A[e];
      B[e] = C{B[e].x + im * a.y, B[e].y - im * a.x};  // + conj(i im) a
    }
    __syncthreads();
  }
  for (int c = 0; c < (ngroups ? 0 : nin); ++c) {
    const C* in = reinterpret_cast<const C*>(ins.p[c]);
    load_tile<R, N, W, ZTile<R, N>::THREADS>(A, in + plane, rstride, nv);
    __syncthreads();
    fft_column<C, N, false, W, 1, CP>(A, col, t, tw);
    for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
      const int row = e / W, cc = e - row * W;
      R re, im;
      spec_coef<R>(sp, first + c, kx0 + cc, iy, row, N, re, im);
      im = -im;  // conjugate multiplier: the transpose of the real operator
      const C a = A[e];
      B[e] = C{B[e].x + re * a.x - im * a.y, B[e].y + re * a.y + im * a.x};
    }
    __syncthreads();
  }
  fft_column<C, N, true, W, 1, CP>(B, col, t, tw);
  store_tile<R, N, W, ZTile<R, N>::THREADS>(out + plane, B, rstride, nv);
}

}  // namespace pmlens
