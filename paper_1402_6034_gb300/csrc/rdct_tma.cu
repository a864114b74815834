// rdct_tma.cu -- tensor maps for TMA staging of the fused kernel (host).
//
// One 2-D map per plane: uint8 elements, dimensions (width, height) in
// pixels, the plane's pitch as the row stride, a 256 x 16-byte box (32 blocks
// of a row pair, the work item of one warp), no swizzle, zeros outside the
// plane.  The encoder is the driver's cuTensorMapEncodeTiled, reached through
// the runtime's driver entry point (no link against the driver library).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "rdct_internal.h"

namespace rdct {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, []() {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == 128, "tensor map size");

bool tma_available() { return encoder() != nullptr; }

bool tma_plane_ok(const JobDesc &j) {
    return (reinterpret_cast<uintptr_t>(j.src) % 16) == 0 && j.src_pitch % 16 == 0 && j.src_pitch > 0 &&
           j.src_pitch < ((int64_t)1 << 40) && j.nbw > 0 && j.nbh > 0;
}

bool tma_encode_plane(const JobDesc &j, unsigned char *map128) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc || !tma_plane_ok(j)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)j.nbw * 8, (cuuint64_t)j.nbh * 8};
    const cuuint64_t strides[1] = {(cuuint64_t)j.src_pitch};
    const cuuint32_t box[2] = {256, 16};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap m;
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(j.src), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    static_assert(sizeof(m) == 128, "tensor map size");
    for (int i = 0; i < 128; ++i) map128[i] = reinterpret_cast<const unsigned char *>(&m)[i];
    return true;
}

}  // namespace rdct
