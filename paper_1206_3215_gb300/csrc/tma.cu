// Host side of the tensor-memory-accelerator staging (tma.cuh): the tensor
// map of a column pass's input array, encoded by the driver's
// cuTensorMapEncodeTiled (looked up once through the runtime, so the library
// does not link the driver library itself).
#include "tma.cuh"

namespace pss {

cudaError_t encode_col_map(CUtensorMap *map, const void *base, int esz, int64_t nx, int64_t ny, int64_t batch, int w,
                           int parts)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    // the driver's encoder, looked up once (thread-safe static initialisation)
    static const Encode encode = []() -> Encode {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<Encode>(fn) : nullptr;
    }();
    if (!encode) return cudaErrorNotSupported;
    if (esz != 8 && esz != 16) return cudaErrorInvalidValue;
    const int64_t r = ny < 256 ? ny : 256;
    const int64_t real = esz / 2;  // bytes of one real
    if (ny % r || (w * esz) % 16 || nx % w || w * 2 > 256 || ny / r > 256 || parts < 1 || (ny / r) % parts)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[4] = {cuuint64_t(2 * nx), cuuint64_t(r), cuuint64_t(ny / r), cuuint64_t(batch)};
    const cuuint64_t strides[3] = {cuuint64_t(nx * esz), cuuint64_t(r * nx * esz), cuuint64_t(ny * nx * esz)};
    const cuuint32_t box[4] = {cuuint32_t(2 * w), cuuint32_t(r), cuuint32_t(ny / r / parts), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult cr = encode(map, real == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                               const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace pss
