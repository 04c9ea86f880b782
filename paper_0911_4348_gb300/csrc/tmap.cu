// TMA tensor maps for the split operand arrays: a 3-D map over [M][n][ld]
// floats (ld = n rounded up to 32) whose box is 32 columns (128-byte swizzle)
// or 16 columns (64-byte swizzle) x `rows` rows x 1 matrix, rows and columns
// beyond n zero-filled (the map's column extent is n, so the padding is not
// fetched). make_tmap_rows16 is the same over FP16 rows of ld16 halves
// (a multiple of 64), box 64 halves (128 bytes) wide; make_tmap_tail16 is the
// 2-D form over [n][pitch] FP16 rows (the first convolution's packed tail).
// The encoder comes from the driver through the runtime's entry-point lookup,
// so no link against libcuda is needed.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace fedvr {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encoder() {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  cudaGetLastError();
}

}  // namespace

cudaError_t make_tmap_rows(CUtensorMap *map, const float *base, int n, int M, int ld,
                           int rows, int box_cols) {
  std::call_once(g_encode_once, load_encoder);
  if (!g_encode) return cudaErrorNotSupported;
  if (rows < 1 || rows > 256 || (ld % 32) != 0 || (box_cols != 32 && box_cols != 16))
    return cudaErrorInvalidValue;
  // columns past n lie outside the map and are zero-filled by the copy engine
  // without being read (the arrays hold zeros there as well)
  const cuuint64_t cols = n >= box_cols ? (cuuint64_t)n : (cuuint64_t)ld;
  const cuuint64_t dims[3] = {cols, (cuuint64_t)n, (cuuint64_t)M};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)n * (cuuint64_t)ld * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_rows16(CUtensorMap *map, const void *base, int n, int M, int ld16,
                             int rows) {
  std::call_once(g_encode_once, load_encoder);
  if (!g_encode) return cudaErrorNotSupported;
  if (rows < 1 || rows > 256 || (ld16 % 64) != 0) return cudaErrorInvalidValue;
  const cuuint64_t cols = n >= 64 ? (cuuint64_t)n : (cuuint64_t)ld16;
  const cuuint64_t dims[3] = {cols, (cuuint64_t)n, (cuuint64_t)M};
  const cuuint64_t strides[2] = {(cuuint64_t)ld16 * 2, (cuuint64_t)n * (cuuint64_t)ld16 * 2};
  const cuuint32_t box[3] = {64, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_tail16(CUtensorMap *map, const void *base, int n, int cols, int pitch,
                             int rows) {
  std::call_once(g_encode_once, load_encoder);
  if (!g_encode) return cudaErrorNotSupported;
  if (rows < 1 || rows > 256 || (pitch % 64) != 0 || cols < 1 || cols > pitch)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace fedvr
