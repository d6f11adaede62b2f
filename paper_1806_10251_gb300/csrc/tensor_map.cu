// TMA descriptors of the population buffers: a 3-D tensor (x, y, plane) whose
// box is one row of all nine planes plus the halo columns of a strip.
#include <cudaTypedefs.h>

#include "stream_collide_x2.cuh"

namespace lbm {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

template <typename ST>
cudaError_t encode(CUtensorMap *map, CUtensorMapDataType dtype, void *base, int nx, int ny, int pitch,
                   long long plane, int box_x)
{
    auto fn = encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(ST), (cuuint64_t)plane * sizeof(ST)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dtype, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename ST>
cudaError_t encode_pair(CUtensorMap *load, CUtensorMap *store, CUtensorMapDataType dtype, void *base, int nx, int ny,
                        int pitch, long long plane)
{
    // load box of the storage type's step kernel: 64-column strips (two cells
    // per lane) for FP32/FP16/BF16, 32-column strips for FP64
    const int box = sizeof(ST) == 8 ? Tile<ST>::BWX : Tile2<ST>::BWX;
    cudaError_t e = encode<ST>(load, dtype, base, nx, ny, pitch, plane, box);
    if (e != cudaSuccess) return e;
    return encode<ST>(store, dtype, base, nx, ny, pitch, plane, WS);
}

}  // namespace

cudaError_t make_tensor_maps(CUtensorMap *load, CUtensorMap *store, int storage, void *base, int nx, int ny,
                             int pitch, long long plane)
{
    switch (storage) {
    case LBM_STORAGE_F16:
        return encode_pair<__half>(load, store, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, nx, ny, pitch, plane);
    case LBM_STORAGE_BF16:
        return encode_pair<__nv_bfloat16>(load, store, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, nx, ny, pitch, plane);
    case LBM_STORAGE_F64:
        return encode_pair<double>(load, store, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, base, nx, ny, pitch, plane);
    default: return encode_pair<float>(load, store, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, nx, ny, pitch, plane);
    }
}

}  // namespace lbm
