// TMA-pipelined column pass of the 3D FFT (y or z axis of a half-spectrum).
//
// A persistent kernel: each block walks the (plane, kx-tile) column tiles
// with stride gridDim.x and keeps two tile buffers in shared memory.  While
// the block transforms tile i in place, the tensor-memory accelerator
// (cp.async.bulk.tensor) already fills the other buffer with tile i + 1, so
// the HBM reads overlap the shared-memory FFT; the result leaves through a
// TMA store (bulk async group) that overlaps the next tile's transform.
//
// The half-spectrum [z][y][P] complex is described to the TMA as a rank-3
// tensor of reals {2P, n, n} (row pitch P complex, plane pitch n P complex);
// a tile is W complex (2W reals, 16-byte multiple) times n rows, moved as
// n / BOXR boxes of at most 256 rows.  A box lands in shared memory in
// row-major order, i.e. as the [row][W] layout of the column FFT.
//
// Every mbarrier wait is bounded: past the bound the block records
// PM_FLAG_TIMEOUT in the error word and returns after draining its own bulk
// stores (the host reports PM_ERR_TIMEOUT).
#pragma once

#include <cuda.h>

#include "fft_impl.cuh"

namespace pmlens {

// Tile shape: half the plain pass's width for n >= 256, one column per thread
// and two resident blocks per SM (measured at n = 512 FP32 against 16-column
// tiles, two columns per thread or three smaller blocks: the pass is bound by
// the latency of the shared-memory stages, so resident warps win).
template <typename R, int N> struct TmaTile {
  static constexpr int W = (N >= 256 && ColTile<R, N>::W >= 4) ? ColTile<R, N>::W / 2 : ColTile<R, N>::W;
  static constexpr int CP = 1;
  static constexpr int THREADS = W / CP * (N / Plan<N>::V);
  static constexpr int MINB = 2;  // resident blocks per SM the register budget is sized for
  static constexpr int BOXR = N < 256 ? N : 256;
  static constexpr int NBOX = N / BOXR;
  static constexpr int TILE_BYTES = N * W * 2 * (int)sizeof(R);
  static constexpr int TW_BYTES = (N * 2 * (int)sizeof(R) + 1023) / 1024 * 1024;
  static constexpr int SMEM = TW_BYTES + 2 * TILE_BYTES + 64;  // + two mbarriers and a flag
  static constexpr int SMEM_DUAL = TW_BYTES + 3 * TILE_BYTES + 64;  // + the second output's work tile
  static_assert(N % BOXR == 0, "box rows");
  static_assert((2 * W * (int)sizeof(R)) % 16 == 0, "TMA inner box extent must be a 16-byte multiple");
  static_assert(TILE_BYTES % 1024 == 0, "tile buffers stay 1024-byte aligned");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase with parity `parity` has completed; false after the
// bound (each try_wait may suspend for a short system-defined interval, so the
// bound is of the order of a second)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(src)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr int PM_FLAG_TIMEOUT = 1;

// ZAXIS: rows are z (box {2W, 1, BOXR}); else rows are y (box {2W, BOXR, 1}).
// Tile ti: plane = ti / ntx (z for the y pass, y for the z pass), kx tile ti % ntx.
//
// DUAL (inverse y pass of the force / PGD x,y components): the input tile
// holds G = IFFT_z(g A); the block writes i k_x IFFT_y(G) in place and
// IFFT_y(i k_y G) through map2 (k_x, k_y = kf times the signed frequency,
// zero on the Nyquist plane), two transforms per tile read.
template <typename R, int N, bool INV, bool ZAXIS, bool DUAL = false>
__global__ void __launch_bounds__(TmaTile<R, N>::THREADS, TmaTile<R, N>::MINB)
k_fft_cols_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map2, int ntx,
               int ntiles, int* __restrict__ err, R kf) {
  using C = typename CT<R>::T;
  using TT = TmaTile<R, N>;
  constexpr int W = TT::W, CP = TT::CP;
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  C* tw = reinterpret_cast<C*>(smem_tma);
  // tile buffer b at smem_tma + TW_BYTES + b * TILE_BYTES, its mbarrier at bar0 + 8 b
  auto buf = [&](int b) { return reinterpret_cast<C*>(smem_tma + TT::TW_BYTES + b * TT::TILE_BYTES); };
  C* work2 = reinterpret_cast<C*>(smem_tma + TT::TW_BYTES + 2 * TT::TILE_BYTES);  // DUAL only
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_tma + TT::TW_BYTES + (DUAL ? 3 : 2) * TT::TILE_BYTES);
  int* ok_word = reinterpret_cast<int*>(bars + 2);
  const uint32_t bar0 = smem_u32(bars);
  auto bar = [&](int b) { return bar0 + 8u * (uint32_t)b; };
  const bool leader = threadIdx.x == 0;
  // bulk tensor copies need 128-byte aligned shared-memory tiles
  if (smem_u32(buf(0)) & 127u) {
    if (leader) atomicOr(err, PM_FLAG_TIMEOUT);
    return;
  }

  auto coords = [&](int ti, int r0, int& c0, int& c1, int& c2) {
    const int plane = ti / ntx, kx0 = (ti - plane * ntx) * W;
    c0 = 2 * kx0;
    c1 = ZAXIS ? plane : r0;
    c2 = ZAXIS ? r0 : plane;
  };
  auto issue_load = [&](int ti, int b) {
    mbar_expect_tx(bar(b), TT::TILE_BYTES);
#pragma unroll
    for (int q = 0; q < TT::NBOX; ++q) {
      int c0, c1, c2;
      coords(ti, q * TT::BOXR, c0, c1, c2);
      tma_load_3d(smem_u32(buf(b)) + q * TT::BOXR * W * (int)sizeof(C), &map, c0, c1, c2, bar(b));
    }
  };

  if (leader) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
    mbar_init(bar(0), 1);
    mbar_init(bar(1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  make_twiddles<C, N>(tw);
  __syncthreads();
  if (leader && blockIdx.x < ntiles) issue_load(blockIdx.x, 0);

  const int col = CP * (threadIdx.x % (W / CP)), t = threadIdx.x / (W / CP);
  int it = 0;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
    const int b = it & 1;
    const int next = ti + gridDim.x;
    if (leader && (DUAL || next < ntiles)) {
      // the other buffer's (and, DUAL, the second work tile's) last bulk store
      // must have read shared memory before it is refilled
      bulk_wait_read0();
      if (next < ntiles) issue_load(next, b ^ 1);
    }
    // the leader polls (bounded) and broadcasts, so that all threads leave together
    if (leader) *ok_word = mbar_wait(bar(b), (it >> 1) & 1) ? 1 : 0;
    __syncthreads();
    if (!*ok_word) {
      if (leader) {
        atomicOr(err, PM_FLAG_TIMEOUT);
        // let the prefetch already in flight land (bounded) before the block exits
        if (next < ntiles) mbar_wait(bar(b ^ 1), ((it + 1) >> 1) & 1);
      }
      break;
    }
    mbar_wait(bar(b), (it >> 1) & 1);  // completed phase: returns at once, acquires the tile per thread
    if constexpr (DUAL) {
      // work2 <- IFFT_y(i k_y G), then buf <- IFFT_y(i k_x G) in place (rows are k_y,
      // columns k_x): the factors are applied as each transform's first stage reads G
      constexpr int h = N / 2;
      const int kx0 = (ti % ntx) * W;
      fft_column_from<C, N, INV, W, 1, CP>(buf(b), work2, col, t, tw, [&](int row, int, C a) {
        const R oy = row == h ? R(0) : kf * (R)(row <= h ? row : row - N);
        return C{-oy * a.y, oy * a.x};
      });
      fft_column_from<C, N, INV, W, 1, CP>(buf(b), buf(b), col, t, tw, [&](int, int c, C a) {
        const int ix = kx0 + c;
        const R ox = ix == h ? R(0) : kf * (R)(ix <= h ? ix : ix - N);
        return C{-ox * a.y, ox * a.x};
      });  // ends with __syncthreads
    } else {
      fft_column<C, N, INV, W, 1, CP>(buf(b), col, t, tw);  // ends with __syncthreads
    }
    fence_proxy_async();  // generic-proxy writes of the tile -> visible to the bulk store
    __syncthreads();
    if (leader) {
#pragma unroll
      for (int q = 0; q < TT::NBOX; ++q) {
        int c0, c1, c2;
        coords(ti, q * TT::BOXR, c0, c1, c2);
        tma_store_3d(&map, c0, c1, c2, smem_u32(buf(b)) + q * TT::BOXR * W * (int)sizeof(C));
        if constexpr (DUAL) tma_store_3d(&map2, c0, c1, c2, smem_u32(work2) + q * TT::BOXR * W * (int)sizeof(C));
      }
      bulk_commit();
    }
  }
  if (leader) bulk_wait0();
}

// ------------------------------------------------------------- force z pass
// Persistent, TMA-pipelined z pass of a force evaluation (OP_FORCE /
// OP_FORCE_PGD): per (y plane, kx tile) column tile, forward z FFT, scale by
// g = (3/2) Om / k^2, inverse for the x,y group (G) and for i k_z g A (F_z);
// with PGD, rescale by the filter ratio and two more inverses (G_p, S_z).
// The next tile's input arrives by TMA while this one is transformed; each
// pass's result leaves by TMA store.  Shared memory: twiddles, two input
// tiles (the current one is transformed in place), one work tile.
template <typename R, int N> struct ZTma {
  static constexpr int W = ZTile<R, N>::W, CP = ZTile<R, N>::CP, THREADS = ZTile<R, N>::THREADS;
  static constexpr int BOXR = N < 256 ? N : 256;
  static constexpr int NBOX = N / BOXR;
  static constexpr int TILE_BYTES = N * W * 2 * (int)sizeof(R);
  static constexpr int TW_BYTES = (N * 2 * (int)sizeof(R) + 1023) / 1024 * 1024;
  static constexpr int SMEM = TW_BYTES + 3 * TILE_BYTES + 64;
  static_assert((2 * W * (int)sizeof(R)) % 16 == 0, "TMA inner box extent must be a 16-byte multiple");
  static_assert(TILE_BYTES % 1024 == 0, "tile buffers stay 1024-byte aligned");
};

struct ZOutMaps { CUtensorMap m[4]; };  // G, F_z, G_p, S_z

template <typename R, int N>
__global__ void __launch_bounds__(ZTma<R, N>::THREADS, 2)
k_zpass_op_tma(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ ZOutMaps outs, int ntx, int ntiles,
               int npass, SpecParams sp, int* __restrict__ err) {
  using C = typename CT<R>::T;
  using ZT = ZTma<R, N>;
  constexpr int W = ZT::W, CP = ZT::CP;

  extern __shared__ __align__(1024) unsigned char smem_zt[];
  C* tw = reinterpret_cast<C*>(smem_zt);
  auto inbuf = [&](int b) { return reinterpret_cast<C*>(smem_zt + ZT::TW_BYTES + b * ZT::TILE_BYTES); };
  C* B = reinterpret_cast<C*>(smem_zt + ZT::TW_BYTES + 2 * ZT::TILE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_zt + ZT::TW_BYTES + 3 * ZT::TILE_BYTES);
  int* ok_word = reinterpret_cast<int*>(bars + 2);
  const uint32_t bar0 = smem_u32(bars);
  auto bar = [&](int b) { return bar0 + 8u * (uint32_t)b; };
  const bool leader = threadIdx.x == 0;
  if (smem_u32(inbuf(0)) & 127u) {
    if (leader) atomicOr(err, PM_FLAG_TIMEOUT);
    return;
  }
  auto issue_load = [&](int ti, int b) {
    const int plane = ti / ntx, kx0 = (ti - plane * ntx) * W;
    mbar_expect_tx(bar(b), ZT::TILE_BYTES);
#pragma unroll
    for (int q = 0; q < ZT::NBOX; ++q)
      tma_load_3d(smem_u32(inbuf(b)) + q * ZT::BOXR * W * (int)sizeof(C), &in_map, 2 * kx0, plane, q * ZT::BOXR,
                  bar(b));
  };
  auto store = [&](const CUtensorMap* m, int ti, const C* src) {
    const int plane = ti / ntx, kx0 = (ti - plane * ntx) * W;
#pragma unroll
    for (int q = 0; q < ZT::NBOX; ++q)
      tma_store_3d(m, 2 * kx0, plane, q * ZT::BOXR, smem_u32(src) + q * ZT::BOXR * W * (int)sizeof(C));
    bulk_commit();
  };
  if (leader) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&in_map)) : "memory");
    mbar_init(bar(0), 1);
    mbar_init(bar(1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  make_twiddles<C, N>(tw);
  __syncthreads();
  if (leader && blockIdx.x < ntiles) issue_load(blockIdx.x, 0);

  const int col = CP * (threadIdx.x % (W / CP)), t = threadIdx.x / (W / CP);
  const R kf = (R)sp.kf;
  constexpr int h = N / 2;
  const R pratio = (R)(sp.pgd_scale / sp.scale);
  int it = 0;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
    const int b = it & 1, next = ti + gridDim.x;
    if (leader) {
      bulk_wait_read0();  // stores of the previous tile have read their tiles
      if (next < ntiles) issue_load(next, b ^ 1);
    }
    if (leader) *ok_word = mbar_wait(bar(b), (it >> 1) & 1) ? 1 : 0;
    __syncthreads();
    if (!*ok_word) {
      if (leader) {
        atomicOr(err, PM_FLAG_TIMEOUT);
        if (next < ntiles) mbar_wait(bar(b ^ 1), ((it + 1) >> 1) & 1);
      }
      break;
    }
    mbar_wait(bar(b), (it >> 1) & 1);
    C* A = inbuf(b);
    const int iy = ti / ntx, kx0 = (ti - iy * ntx) * W;
    const int fy = iy <= h ? iy : iy - N;
    fft_column<C, N, false, W, 1, CP>(A, col, t, tw);
    for (int pass = 0; pass < npass; ++pass) {
      const bool zc = pass & 1, pg = pass >= 2;
      const bool last = pass == npass - 1;
      C* T = last ? A : B;
      if (!last) {
        // B is the previous pass's store source: wait until the copy engine has read it
        if (leader) bulk_wait_read0();
        __syncthreads();
      }
      // this output's operator, applied as the inverse transform's first stage reads the
      // spectrum A: g = (3/2) Om / k^2 (x,y group G and, times i k_z, F_z); with PGD the
      // filter ratio on top (G_p, S_z).  A itself stays the forward spectrum.
      auto op = [&](int row, int c, C a) {
        const int ix = kx0 + c;
        const int fx = ix <= h ? ix : ix - N, fz = row <= h ? row : row - N;
        const R k2 = kf * kf * (R)(fx * fx + fy * fy + fz * fz);
        const R inv = k2 > R(0) ? R(1) / k2 : R(0);
        R f = (R)sp.scale * inv;
        if (pg) f = k2 > R(0) ? f * pratio * pgd_filter<R>(sp, k2, inv) : R(0);
        if (!zc) return C{f * a.x, f * a.y};
        const R oz = row == h ? R(0) : kf * (R)fz;
        return C{-oz * f * a.y, oz * f * a.x};  // i k_z f a
      };
      fft_column_from<C, N, true, W, 1, CP>(A, T, col, t, tw, op);  // ends with __syncthreads
      fence_proxy_async();
      __syncthreads();
      if (leader) store(&outs.m[pass], ti, T);
    }
  }
  if (leader) bulk_wait0();
}

// Host side: rank-3 tensor map over a half-spectrum buffer for the column pass
// of axis `zaxis` (false: y rows).  Returns false if the driver rejects it.
bool make_cols_map(CUtensorMap* map, void* base, int n, int P, int w, int boxr, bool zaxis, bool dbl);

}  // namespace pmlens
