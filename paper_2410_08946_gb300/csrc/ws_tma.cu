// ws_tma.cu -- host-side encoding of TMA tensor maps (CUtensorMap) through
// the CUDA driver entry point, so that the library does not link libcuda.
#include <mutex>

#include "ws_tma.cuh"

namespace ws {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

bool make_tmap_3d(CUtensorMap *map, const void *base, int elem, uint64_t W, uint64_t H, uint64_t D, uint32_t bx,
                  uint32_t by, uint32_t bz)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if (((uintptr_t)base & 15) != 0) return false;
    if ((W * elem) % 16 != 0 || (bx * elem) % 16 != 0) return false;
    if (bx > 256 || by > 256 || bz > 256) return false;
    CUtensorMapDataType dt = elem == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                       : (elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_INT32);
    cuuint64_t dims[3] = {W, H, D};
    cuuint64_t strides[2] = {W * elem, W * H * elem};
    cuuint32_t box[3] = {bx, by, bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace ws
