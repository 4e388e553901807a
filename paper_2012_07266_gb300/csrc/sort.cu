// Spatial reordering of the particle state.
//
// Particles start in Lagrangian (lattice) order; as they cluster, consecutive
// particles no longer sit in neighbouring cells and the CIC gathers/scatters of
// a step re-fetch mesh lines from HBM several times.  Every few steps the state
// is counting-sorted by coarse block of 8^3 force-mesh cells (row-major block
// order): count, exclusive scan, scatter into the second state buffer.  (A
// Morton block order, which keeps a thread block's run of particles in a
// compact region, measured 10% less DRAM traffic in kick-drift-paint but a 12%
// slower launch at pm256, so row-major order stays.)  The original index of
// each particle travels along (pid), so outputs and the initial-condition
// adjoint stay in lattice order.
#include <algorithm>

#include "pm_internal.h"
#include "warp_agg.cuh"

namespace pmlens {
namespace {

constexpr int kBlk = 8;  // cells per bucket side

__device__ __forceinline__ unsigned bucket_of(uint32_t c, int nbs) {
  const unsigned ix = c & 1023u, iy = (c >> 10) & 1023u, iz = c >> 20;
  return ((iz / kBlk) * nbs + iy / kBlk) * nbs + ix / kBlk;
}

inline long long buckets_per_side(int M) { return (M + kBlk - 1) / kBlk; }

__global__ void __launch_bounds__(256) k_bucket_count(const uint32_t* __restrict__ cell, long long np, int nbs,
                                                      unsigned* __restrict__ count) {
  __shared__ unsigned wsm[256];
  unsigned* ws = wsm + (threadIdx.x & ~31);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); j0 < np; j0 += stride) {
    const long long j = j0 + (threadIdx.x & 31);
    const bool valid = j < np;
    const unsigned b = bucket_of(cell[valid ? j : np - 1], nbs);
    warp_agg_add(count, b, valid ? 1u : 0u, ws);
  }
}

// exclusive scan of n counts: per-block scan of 1024 entries, then the block totals
__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned* __restrict__ in, unsigned* __restrict__ out,
                                                      unsigned* __restrict__ totals, long long n) {
  __shared__ unsigned s[1024];
  const long long i = blockIdx.x * 1024LL + threadIdx.x;
  const unsigned v = i < n ? in[i] : 0u;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned t = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) totals[blockIdx.x] = s[1023];
}

// one block: exclusive scan of the block totals in place (nt <= 4096)
__global__ void __launch_bounds__(1024) k_scan_totals(unsigned* __restrict__ totals, int nt) {
  __shared__ unsigned s[4096];
  for (int i = threadIdx.x; i < 4096; i += 1024) s[i] = i < nt ? totals[i] : 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned acc = 0;
    for (int i = 0; i < nt; ++i) {
      const unsigned v = s[i];
      s[i] = acc;
      acc += v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nt; i += 1024) totals[i] = s[i];
}

__global__ void k_scan_add(unsigned* __restrict__ out, const unsigned* __restrict__ totals, long long n) {
  const long long i = blockIdx.x * 1024LL + threadIdx.x;
  if (i < n) out[i] += totals[blockIdx.x];
}

template <typename R>
struct SortIO {
  const uint32_t* cell;
  const R* frac;
  const R* mom;
  const uint32_t* pid;
  uint32_t* cell2;
  R* frac2;
  R* mom2;
  uint32_t* pid2;
};

// each particle takes the next slot of its bucket: the lanes of a warp that
// share a bucket reserve their slots with one atomic
template <typename R>
__global__ void __launch_bounds__(256) k_bucket_scatter(SortIO<R> io, long long np, int nbs,
                                                        unsigned* __restrict__ cursor) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); j0 < np; j0 += stride) {
    const long long j = j0 + lane;
    const bool valid = j < np;
    const long long jj = valid ? j : np - 1;
    const uint32_t c = io.cell[jj];
    const unsigned b = valid ? bucket_of(c, nbs) : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (lane == leader && valid) base = atomicAdd(cursor + b, (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) continue;
    const unsigned dst = base + __popc(peers & ((1u << lane) - 1u));
    io.cell2[dst] = c;
    io.pid2[dst] = io.pid[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      io.frac2[dst + d * np] = io.frac[j + d * np];
      io.mom2[dst + d * np] = io.mom[j + d * np];
    }
  }
}

__global__ void k_iota(uint32_t* __restrict__ p, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    p[j] = (uint32_t)j;
}

// dst[pid[j]] = src[j] for 3 components of n (to lattice order)
template <typename R>
__global__ void k_unpermute3(const R* __restrict__ src, const uint32_t* __restrict__ pid, R* __restrict__ dst,
                             long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const long long o = pid[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) dst[o + d * n] = src[j + d * n];
  }
}

// dst[j] = src[pid[j]] for 3 components (from lattice order)
template <typename R>
__global__ void k_permute3(const R* __restrict__ src, const uint32_t* __restrict__ pid, R* __restrict__ dst,
                           long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const long long o = pid[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) dst[j + d * n] = src[o + d * n];
  }
}

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

void launch_iota(pm_ctx* c) {
  ProfScope ps(&c->prof, KK_MISC, c->stream, 4.0 * c->np);
  k_iota<<<gridn(c->np), 256, 0, c->stream>>>(reinterpret_cast<uint32_t*>(c->ws + c->L.pid), c->np);
}

template <typename R>
cudaError_t sort_particles(pm_ctx* c) {
  const int nbs = (int)buckets_per_side(c->M);
  const long long nb = (long long)nbs * nbs * nbs;
  unsigned* count = reinterpret_cast<unsigned*>(c->ws + c->L.sort_cnt);
  unsigned* offs = count + nb;
  unsigned* tot = offs + nb;
  cudaStream_t s = c->stream;
  ProfScope ps(&c->prof, KK_MISC, s, c->np * (4.0 + 2.0 * (8.0 + 6.0 * sizeof(R))));
  cudaError_t e = cudaMemsetAsync(count, 0, nb * sizeof(unsigned), s);
  if (e) return e;
  k_bucket_count<<<gridn(c->np), 256, 0, s>>>(reinterpret_cast<const uint32_t*>(c->ws + c->L.cell), c->np, nbs,
                                               count);
  const int nblk = (int)((nb + 1023) / 1024);
  k_scan_blocks<<<nblk, 1024, 0, s>>>(count, offs, tot, nb);
  k_scan_totals<<<1, 1024, 0, s>>>(tot, nblk);
  k_scan_add<<<nblk, 1024, 0, s>>>(offs, tot, nb);
  SortIO<R> io;
  io.cell = reinterpret_cast<const uint32_t*>(c->ws + c->L.cell);
  io.frac = reinterpret_cast<const R*>(c->ws + c->L.frac);
  io.mom = reinterpret_cast<const R*>(c->ws + c->L.mom);
  io.pid = reinterpret_cast<const uint32_t*>(c->ws + c->L.pid);
  io.cell2 = reinterpret_cast<uint32_t*>(c->ws + c->L.cell2);
  io.frac2 = reinterpret_cast<R*>(c->ws + c->L.frac2);
  io.mom2 = reinterpret_cast<R*>(c->ws + c->L.mom2);
  io.pid2 = reinterpret_cast<uint32_t*>(c->ws + c->L.pid2);
  k_bucket_scatter<R><<<gridn(c->np), 256, 0, s>>>(io, c->np, nbs, offs);
  if ((e = cudaGetLastError())) return e;
  std::swap(c->L.cell, c->L.cell2);
  std::swap(c->L.frac, c->L.frac2);
  std::swap(c->L.mom, c->L.mom2);
  std::swap(c->L.pid, c->L.pid2);
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_unpermute3(pm_ctx* c, const R* src, const uint32_t* pid, R* dst) {
  ProfScope ps(&c->prof, KK_MISC, c->stream, c->np * (4.0 + 6.0 * sizeof(R)));
  k_unpermute3<R><<<gridn(c->np), 256, 0, c->stream>>>(src, pid, dst, c->np);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_permute3(pm_ctx* c, const R* src, const uint32_t* pid, R* dst) {
  ProfScope ps(&c->prof, KK_MISC, c->stream, c->np * (4.0 + 6.0 * sizeof(R)));
  k_permute3<R><<<gridn(c->np), 256, 0, c->stream>>>(src, pid, dst, c->np);
  return cudaGetLastError();
}

size_t sort_scratch_bytes(int M) {
  const long long nbs = buckets_per_side(M);
  const long long nb = nbs * nbs * nbs;
  return (size_t)(2 * nb + (nb + 1023) / 1024 + 1024) * sizeof(unsigned);
}

#define PM_SORT_INST(R)                                                          \
  template cudaError_t sort_particles<R>(pm_ctx*);                              \
  template cudaError_t launch_unpermute3<R>(pm_ctx*, const R*, const uint32_t*, R*); \
  template cudaError_t launch_permute3<R>(pm_ctx*, const R*, const uint32_t*, R*);
PM_SORT_INST(float)
PM_SORT_INST(double)

}  // namespace pmlens
