// Host helpers: TMA tensor maps of the voltage and weight operands (K-major,
// 128-byte swizzle), encoded through the driver entry point fetched once.
#include <mutex>

#include "tmap.h"

namespace bfi {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static bool encode3(CUtensorMap *m, const void *ptr, cuuint64_t d0, cuuint64_t d1, cuuint64_t d2, int es, int box0,
                    int box1, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = es == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {d0 * es, d0 * d1 * es};
    cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_voltage_map(CUtensorMap *m, const void *x, int two_n, int T, int C, int es, int ke, int nt)
{
    return encode3(m, x, (cuuint64_t)two_n, (cuuint64_t)T, (cuuint64_t)C, es, ke, nt);
}

bool encode_weight_map(CUtensorMap *m, const void *w, int k_pad, int m_pad, int C, int es, int ke)
{
    return encode3(m, w, (cuuint64_t)k_pad, (cuuint64_t)m_pad, (cuuint64_t)C, es, ke, kRowsPerMTile);
}

bool encode_raw_map(CUtensorMap *m, const void *x, int row_bytes, int T, int C, int box_bytes, int nt)
{
    return encode3(m, x, (cuuint64_t)row_bytes, (cuuint64_t)T, (cuuint64_t)C, 1, box_bytes, nt,
                   CU_TENSOR_MAP_SWIZZLE_NONE);
}

}  // namespace bfi
