// Host-side tensor maps for the TMA-pipelined column passes.  The driver's
// cuTensorMapEncodeTiled is reached through the runtime's entry-point query,
// so the library needs no link-time dependency on the driver library.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace pmlens {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

// Half-spectrum [n][n][P] complex as a rank-3 tensor of reals {2P, n, n}:
// dimension 1 (y) has pitch P complex, dimension 2 (z) pitch n P complex.
// The box is {2w, boxr, 1} for the y pass and {2w, 1, boxr} for the z pass.
// Requirements checked by the driver: base 16-byte aligned, pitches 16-byte
// multiples, 2w reals a 16-byte multiple, box extents <= 256.
bool make_cols_map(CUtensorMap* map, void* base, int n, int P, int w, int boxr, bool zaxis, bool dbl) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t es = dbl ? 8 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * P, (cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t pitch[2] = {(cuuint64_t)2 * P * es, (cuuint64_t)2 * P * es * (cuuint64_t)n};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * w), (cuuint32_t)(zaxis ? 1 : boxr), (cuuint32_t)(zaxis ? boxr : 1)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                         pitch, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace pmlens
