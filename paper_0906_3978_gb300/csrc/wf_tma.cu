// wf_tma.cu -- host side of the tensor copies: tensor maps over packed half spectra, encoded
// through the runtime's driver entry point (the library does not link libcuda itself).
#include <cudaTypedefs.h>

#include <mutex>

#include "wf_tma.cuh"

namespace wf {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  });
  return fn;
}

bool make_spectrum_map(CUtensorMap* map, void* base, int n, int nb, bool fp64, int nl, int b1, int b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc || !base || n <= 0 || nb <= 0) return false;
  const cuuint64_t es = fp64 ? 8 : 4;  // bytes of one real component
  const cuuint64_t nh = (cuuint64_t)n / 2;
  const cuuint64_t dims[4] = {2 * nh, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nb};
  const cuuint64_t strides[3] = {2 * nh * es, (cuuint64_t)n * 2 * nh * es, (cuuint64_t)n * n * 2 * nh * es};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * nl), (cuuint32_t)b1, (cuuint32_t)b2, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(map, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace wf
