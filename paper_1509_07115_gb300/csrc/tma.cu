// tma.cu -- TMA tensor-map encoding (driver entry point fetched at run time so
// the library does not link libcuda directly).
#include <cudaTypedefs.h>

#include <mutex>

#include "plan.cuh"

namespace dsbt {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static void load_encode() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

int encode_tmap_f32_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols) {
    std::call_once(g_encode_once, load_encode);
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DSBT_ERR_CUDA;
    }
    // base 16-byte aligned, row stride a multiple of 16 bytes, inner box 128 bytes
    if (((uintptr_t)base & 15) != 0 || (cols * 4) % 16 != 0 || box_cols * 4 != 128 || box_rows > 256) {
        set_error("tensor map: alignment or box constraint violated");
        return DSBT_ERR_INVALID;
    }
    cuuint64_t gdim[2] = {cols, rows};
    cuuint64_t gstride[1] = {cols * 4};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), gdim,
                          gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DSBT_ERR_CUDA;
    }
    return DSBT_OK;
}

int encode_tmap_f16_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols) {
    std::call_once(g_encode_once, load_encode);
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DSBT_ERR_CUDA;
    }
    // base 16-byte aligned, row stride a multiple of 16 bytes, inner box 128 bytes
    if (((uintptr_t)base & 15) != 0 || (cols * 2) % 16 != 0 || box_cols * 2 != 128 || box_rows > 256) {
        set_error("tensor map: alignment or box constraint violated");
        return DSBT_ERR_INVALID;
    }
    cuuint64_t gdim[2] = {cols, rows};
    cuuint64_t gstride[1] = {cols * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), gdim,
                          gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DSBT_ERR_CUDA;
    }
    return DSBT_OK;
}

}  // namespace dsbt
