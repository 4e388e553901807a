// PM forces without any device allocation: the scratch meshes of the force
// computation (density, half-spectrum, three spectral outputs, three force
// meshes) live in one file-scope __device__ array instead of a workspace.
//
// For callers that cannot allocate device memory themselves: code running
// inside a host framework whose allocator owns the device memory, plugins or
// callbacks that must not allocate, processes under a hard device-memory
// budget.  The array is sized for meshes up to kStaticMaxMesh^3 (FP32) and
// every GPU that loads this library holds it until the process exits.
#include <mutex>

#include "pm_internal.h"

namespace pmlens {
namespace {

constexpr int kStaticMaxMesh = 64;
constexpr int kStaticMaxP = 48;  // padded half-spectrum row pitch of a 64 mesh
constexpr size_t kRealBytes = (size_t)kStaticMaxMesh * kStaticMaxMesh * kStaticMaxMesh * sizeof(float);
constexpr size_t kCplxBytes = (size_t)kStaticMaxMesh * kStaticMaxMesh * kStaticMaxP * sizeof(float2);
constexpr size_t kStaticBytes = 4 * kRealBytes + 4 * kCplxBytes;  // rho, F x3, cbuf, spectral outputs x3

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
void* g_scratch_addr[64] = {};

// device address of the scratch array on the current device (looked up once
// per device; the host-side symbol itself is not a device address).  The
// first lookup on a device loads the module there if no kernel of the library
// has run on it yet (lazy loading); the cached address is stale after a
// cudaDeviceReset, after which this entry point must not be used.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__device__ __forceinline__ void cell_frac(double x, double cpl, int M, int& i, float& f) {
  const double X = x * cpl;
  const double fl = floor(X);
  float fr = (float)(X - fl);
  long long ii = (long long)fl;
  if (fr >= 1.f) { fr = 0.f; ii += 1; }
  long long r = ii % M;
  i = (int)(r < 0 ? r + M : r);
  f = fr;
}

__global__ void k_static_paint(const double* __restrict__ x, long long n, int M, double cpl, float mass,
                               float* __restrict__ rho) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    int i[3];
    float f[3];
    for (int d = 0; d < 3; ++d) cell_frac(x[3 * j + d], cpl, M, i[d], f[d]);
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
      const int ix = (i[0] + dx) % M, iy = (i[1] + dy) % M, iz = (i[2] + dz) % M;
      const float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
      atomicAdd(rho + ((long long)iz * M + iy) * M + ix, mass * w);
    }
  }
}

__global__ void k_static_readout(const double* __restrict__ x, long long n, int M, double cpl, double scale,
                                 const float* __restrict__ F, double* __restrict__ out) {
  const long long m3 = (long long)M * M * M;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    int i[3];
    float f[3];
    for (int d = 0; d < 3; ++d) cell_frac(x[3 * j + d], cpl, M, i[d], f[d]);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
      const int ix = (i[0] + dx) % M, iy = (i[1] + dy) % M, iz = (i[2] + dz) % M;
      const float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
      const long long o = ((long long)iz * M + iy) * M + ix;
      for (int k = 0; k < 3; ++k) acc[k] += w * F[k * m3 + o];
    }
    for (int k = 0; k < 3; ++k) out[3 * j + k] = scale * (double)acc[k];
  }
}

}  // namespace
}  // namespace pmlens

using namespace pmlens;

extern "C" pm_status pm_forces_static(const double* d_x, int64_t n, int32_t nmesh, double box, double omega_m,
                                      double* d_f, void* stream) {
  if (!d_x || !d_f || n < 1 || !(box > 0) || !(omega_m > 0)) return PM_ERR_ARG;
  if (nmesh > kStaticMaxMesh || !fft_supported(nmesh)) return PM_ERR_UNSUPPORTED;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PM_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int M = nmesh;
  const int P = (M / 2 + 1 + 15) / 16 * 16;
  char* b = reinterpret_cast<char*>(base);
  float* rho = reinterpret_cast<float*>(b);
  float* F = reinterpret_cast<float*>(b + kRealBytes);  // three meshes
  void* cbuf = b + 4 * kRealBytes;
  void* ub[3] = {b + 4 * kRealBytes + kCplxBytes, b + 4 * kRealBytes + 2 * kCplxBytes,
                 b + 4 * kRealBytes + 3 * kCplxBytes};
  const long long m3 = (long long)M * M * M;
  float* outs[3] = {F, F + m3, F + 2 * m3};
  // the array keeps the previous call's contents: the density must start at zero
  if (cudaMemsetAsync(rho, 0, m3 * sizeof(float), s) != cudaSuccess) return PM_ERR_CUDA;
  const double cpl = M / box;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_static_paint<<<(int)blocks, 256, 0, s>>>(d_x, n, M, cpl, (float)((double)m3 / (double)n), rho);
  SpecParams sp = {};
  sp.op = OP_FORCE;
  sp.kf = 2.0 * M_PI / box;
  sp.scale = 1.5 * omega_m * cpl / (double)m3;
  if (spectral_apply<float>(rho, cbuf, ub, outs, 3, M, P, sp, s, nullptr) != cudaSuccess) return PM_ERR_CUDA;
  k_static_readout<<<(int)blocks, 256, 0, s>>>(d_x, n, M, cpl, box / M, F, d_f);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}
