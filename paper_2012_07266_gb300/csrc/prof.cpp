// Launch counting and optional CUDA-event timing of the library's kernels.
#include "pm_internal.h"

namespace pmlens {

const char* kernel_kind_name(int k) {
  static const char* names[KK_COUNT] = {"kick_drift_paint", "paint", "fft_x_r2c", "fft_y_fwd", "fft_z_fwd",
                                        "fft_z_spectral_op", "fft_y_inv", "fft_x_c2r", "lens_project", "ic",
                                        "misc", "adjoint_particles", "adjoint_spectral", "adjoint_lens",
                                        "tangent", "adjoint_paint", "adjoint_readout"};
  return (k >= 0 && k < KK_COUNT) ? names[k] : "unknown";
}

cudaEvent_t Prof::get() {
  if (used == pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[used++];
}

void Prof::resolve() {
  for (const Rec& r : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.kind] += t;
      timed[r.kind] += 1;
    }
  }
  pending.clear();
  used = 0;
}

Prof::~Prof() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

ProfScope::ProfScope(Prof* p_, int k, cudaStream_t s_, double algo_bytes) : p(p_), kind(k), s(s_) {
  if (!p) return;
  p->launches[kind] += 1;
  p->bytes[kind] += algo_bytes;
  if (p->timing) {
    a = p->get();
    if (a) cudaEventRecord(a, s);
  }
}

ProfScope::~ProfScope() {
  if (!p || !p->timing || !a) return;
  cudaEvent_t b = p->get();
  if (!b) return;
  cudaEventRecord(b, s);
  p->pending.push_back(Prof::Rec{kind, a, b});
}

}  // namespace pmlens
