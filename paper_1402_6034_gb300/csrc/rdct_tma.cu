// rdct_tma.cu -- tensor maps for TMA staging of the fused kernel (host).
//
// Two 2-D maps per plane, for the source and the reconstruction: uint8
// elements, dimensions (width, height) in pixels, the plane's pitch as the row
// stride, a 256 x 16-byte box (32 blocks of a row pair, the work item of one
// warp), no swizzle; loads read zeros outside the plane, stores drop what
// falls outside it.  The encoder is the driver's cuTensorMapEncodeTiled, reached through
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

namespace {

bool aligned16(const void *p, int64_t pitch) {
    return (reinterpret_cast<uintptr_t>(p) % 16) == 0 && pitch % 16 == 0 && pitch > 0 && pitch < ((int64_t)1 << 40);
}

bool encode_2d(const void *base, int64_t w, int64_t h, int64_t pitch, unsigned char *map128) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc || !aligned16(base, pitch) || w <= 0 || h <= 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {256, 16};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap m;
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    for (int i = 0; i < 128; ++i) map128[i] = reinterpret_cast<const unsigned char *>(&m)[i];
    return true;
}

}  // namespace

bool tma_plane_ok(const JobDesc &j) {
    return aligned16(j.src, j.src_pitch) && (j.dst == nullptr || aligned16(j.dst, j.dst_pitch)) && j.nbw > 0 &&
           j.nbh > 0;
}

bool tma_encode_plane(const JobDesc &j, unsigned char *maps256) {
    if (!tma_plane_ok(j)) return false;
    for (int i = 0; i < 256; ++i) maps256[i] = 0;
    if (!encode_2d(j.src, (int64_t)j.nbw * 8, (int64_t)j.nbh * 8, j.src_pitch, maps256)) return false;
    return j.dst == nullptr || encode_2d(j.dst, (int64_t)j.nbw * 8, (int64_t)j.nbh * 8, j.dst_pitch, maps256 + 128);
}

}  // namespace rdct
