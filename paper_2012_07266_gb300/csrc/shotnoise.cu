// Binned flat-sky angular power spectrum of convergence maps (Sec. 4,
// Fig. accuracy: the spectra of the simulated maps and of the shot-noise runs
// whose average is subtracted from them).
//
// For an n x n map (n a power of two, FP64 throughout):
//   C(m) = Omega_pix |DFT(kappa)(m)|^2 / n^2,  l(m) = (2 pi / FOV) |m|,
// averaged over the modes of each bin edges[b] <= l < edges[b+1].  Three
// kernels per map: a row FFT that stores its result transposed, a column FFT
// fused with the binning (each CTA accumulates its column's modes in shared
// memory and adds them to the global bins once), and one final combine of all
// maps, d_cl = beta d_cl + alpha (sum / count).  The 2D DFT is separable, and
// the transposed intermediate only swaps m_x and m_y, which |m| does not see.
// Each FFT runs in shared memory on one row: the input is loaded in
// bit-reversed order and log2(n) radix-2 decimation-in-time stages run in
// place, with twiddles exp(-2 pi i j / n) from a table built once per call.
// Maps are small next to the particle work (a 2048^2 map is 32 MB), so the
// kernels aim at simplicity; the transposed store is the only strided access.
#include <cmath>
#include <cstring>

#include "pm_internal.h"

namespace {

constexpr int kClThreads = 256;
constexpr int kClMaxBins = 2048;
constexpr int kClMaxLog = 12;  // n <= 4096

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct ClLayout {
  size_t work, tw, edges, sums, counts, total;
};

ClLayout cl_layout(int n, int nmaps, int nbins) {
  ClLayout L;
  size_t o = 0;
  L.work = o;   o += align256((size_t)n * n * sizeof(double2));
  L.tw = o;     o += align256((size_t)(n / 2) * sizeof(double2));
  L.edges = o;  o += align256((size_t)(nbins + 1) * sizeof(double));
  L.sums = o;   o += align256((size_t)nmaps * nbins * sizeof(double));
  L.counts = o; o += align256((size_t)nbins * sizeof(unsigned long long));
  L.total = o;
  return L;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_cl_twiddles(double2* __restrict__ tw, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n / 2; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * j / n, &sn, &cs);  // 2j/n exact for n a power of two
    tw[j] = make_double2(cs, -sn);
  }
}

// in-place radix-2 DIT FFT of a[0..n) (already in bit-reversed order)
__device__ void fft_inplace(double2* a, int n, const double2* __restrict__ tw) {
  for (int h = 1; h < n; h <<= 1) {
    const int stride = n / (2 * h);
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int k = t & (h - 1);
      const int i0 = 2 * (t - k) + k, i1 = i0 + h;
      const double2 wb = cmul(tw[k * stride], a[i1]);
      const double2 u = a[i0];
      a[i0] = make_double2(u.x + wb.x, u.y + wb.y);
      a[i1] = make_double2(u.x - wb.x, u.y - wb.y);
    }
    __syncthreads();
  }
}

// row iy of the map -> its DFT along x, stored as column iy of work (work[mx][iy])
__global__ void __launch_bounds__(kClThreads) k_cl_rows(const double* __restrict__ map, double2* __restrict__ work,
                                                        const double2* __restrict__ tw, int n, int logn) {
  extern __shared__ double2 a[];
  const int r = blockIdx.x;
  const double* row = map + (size_t)r * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) a[__brev(j) >> (32 - logn)] = make_double2(row[j], 0.0);
  __syncthreads();
  fft_inplace(a, n, tw);
  for (int k = threadIdx.x; k < n; k += blockDim.x) work[(size_t)k * n + r] = a[k];
}

// row mx of work -> the DFT along y; each mode's power into its bin
__global__ void __launch_bounds__(kClThreads) k_cl_cols(const double2* __restrict__ work,
                                                        const double2* __restrict__ tw,
                                                        const double* __restrict__ edges, int nbins, int n, int logn,
                                                        double lscale, double pscale, double* __restrict__ sums,
                                                        unsigned long long* __restrict__ counts) {
  extern __shared__ double2 a[];
  double* e = reinterpret_cast<double*>(a + n);
  double* bsum = e + nbins + 1;
  unsigned int* bcnt = reinterpret_cast<unsigned int*>(bsum + nbins);
  const int k = blockIdx.x;
  const double2* row = work + (size_t)k * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) a[__brev(j) >> (32 - logn)] = row[j];
  for (int b = threadIdx.x; b <= nbins; b += blockDim.x) e[b] = edges[b];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    bsum[b] = 0.0;
    bcnt[b] = 0u;
  }
  __syncthreads();
  fft_inplace(a, n, tw);
  const int mx = k < n / 2 ? k : k - n;
  const double lo = e[0], hi = e[nbins];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int my = j < n / 2 ? j : j - n;
    const double l = lscale * sqrt((double)(mx * mx + my * my));
    if (!(l >= lo) || !(l < hi)) continue;
    int b0 = 0, b1 = nbins;  // e[b0] <= l < e[b1]
    while (b1 - b0 > 1) {
      const int mid = (b0 + b1) >> 1;
      if (l >= e[mid]) b0 = mid; else b1 = mid;
    }
    const double2 v = a[j];
    atomicAdd(&bsum[b0], pscale * (v.x * v.x + v.y * v.y));
    atomicAdd(&bcnt[b0], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    if (!bcnt[b]) continue;
    atomicAdd(&sums[b], bsum[b]);
    if (counts) atomicAdd(&counts[b], (unsigned long long)bcnt[b]);
  }
}

__global__ void k_cl_combine(const double* __restrict__ sums, const unsigned long long* __restrict__ counts,
                             int nmaps, int nbins, double alpha, double beta, double* __restrict__ cl) {
  const int tot = nmaps * nbins;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    const unsigned long long c = counts[i % nbins];
    const double v = c ? sums[i] / (double)c : 0.0;
    cl[i] = (beta == 0.0 ? 0.0 : beta * cl[i]) + alpha * v;
  }
}

int ilog2_pow2(int n) {
  if (n <= 0 || (n & (n - 1))) return -1;
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

bool cl_args_ok(int npix, int nmaps, int nbins) {
  const int logn = ilog2_pow2(npix);
  return logn >= 3 && logn <= kClMaxLog && nmaps >= 1 && nbins >= 1 && nbins <= kClMaxBins;
}

}  // namespace

extern "C" {

pm_status pm_map_cl_workspace_size(int32_t npix, int32_t nmaps, int32_t nbins, size_t* bytes) {
  if (!bytes || !cl_args_ok(npix, nmaps, nbins)) return PM_ERR_ARG;
  *bytes = cl_layout(npix, nmaps, nbins).total;
  return PM_OK;
}

pm_status pm_map_cl(const double* d_maps, int32_t nmaps, int32_t npix, double fov_deg, const double* h_edges,
                    int32_t nbins, double alpha, double beta, double* d_cl, int64_t* h_counts, void* d_workspace,
                    size_t workspace_bytes, void* stream) {
  if (!d_maps || !h_edges || !d_cl || !d_workspace || !cl_args_ok(npix, nmaps, nbins)) return PM_ERR_ARG;
  if (!(fov_deg > 0.0) || !std::isfinite(fov_deg) || !std::isfinite(alpha) || !std::isfinite(beta))
    return PM_ERR_ARG;
  for (int b = 0; b <= nbins; ++b) {
    if (std::isnan(h_edges[b])) return PM_ERR_ARG;
    if (b > 0 && !(h_edges[b] > h_edges[b - 1])) return PM_ERR_ARG;
  }
  const ClLayout L = cl_layout(npix, nmaps, nbins);
  if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) return PM_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(d_workspace);
  double2* work = reinterpret_cast<double2*>(ws + L.work);
  double2* tw = reinterpret_cast<double2*>(ws + L.tw);
  double* edges = reinterpret_cast<double*>(ws + L.edges);
  double* sums = reinterpret_cast<double*>(ws + L.sums);
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(ws + L.counts);
  const int n = npix, logn = ilog2_pow2(npix);
  // l of a mode: (2 pi / FOV_rad) sqrt(mx^2 + my^2), FOV_rad = fov_deg (pi / 180), in this order
  const double fov_rad = fov_deg * (M_PI / 180.0);
  const double lscale = 2.0 * M_PI / fov_rad;
  const double opix = (fov_rad / n) * (fov_rad / n);
  const double pscale = opix / ((double)n * (double)n);
  const size_t smem_rows = (size_t)n * sizeof(double2);
  const size_t smem_cols = smem_rows + (size_t)(2 * nbins + 1) * sizeof(double) + (size_t)nbins * sizeof(unsigned int);
  if (cudaFuncSetAttribute(k_cl_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows) ||
      cudaFuncSetAttribute(k_cl_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols))
    return PM_ERR_CUDA;
  if (cudaMemcpyAsync(edges, h_edges, (size_t)(nbins + 1) * sizeof(double), cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(sums, 0, (size_t)nmaps * nbins * sizeof(double), s) ||
      cudaMemsetAsync(counts, 0, (size_t)nbins * sizeof(unsigned long long), s))
    return PM_ERR_CUDA;
  k_cl_twiddles<<<(n / 2 + 255) / 256, 256, 0, s>>>(tw, n);
  for (int m = 0; m < nmaps; ++m) {
    k_cl_rows<<<n, kClThreads, smem_rows, s>>>(d_maps + (size_t)m * n * n, work, tw, n, logn);
    k_cl_cols<<<n, kClThreads, smem_cols, s>>>(work, tw, edges, nbins, n, logn, lscale, pscale,
                                               sums + (size_t)m * nbins, m == 0 ? counts : nullptr);
  }
  const int tot = nmaps * nbins;
  k_cl_combine<<<(tot + 255) / 256, 256, 0, s>>>(sums, counts, nmaps, nbins, alpha, beta, d_cl);
  if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
  if (h_counts) {
    if (cudaMemcpyAsync(h_counts, counts, (size_t)nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return PM_ERR_CUDA;
  }
  return PM_OK;
}

}  // extern "C"
