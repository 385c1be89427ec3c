// tma_host.cuh -- host side of the TMA loads: tensor-map descriptors of padded
// 3D fields (x fastest), encoded through the driver entry point.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cspht {

inline PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// Descriptor of one padded field of grid G with a (bw x bh x 1) box.
template <typename T>
inline bool make_tmap(CUtensorMap *m, const T *base, const Grid &G, int bw, int bh) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)G.px, (cuuint64_t)G.py, (cuuint64_t)G.pz};
    cuuint64_t strides[2] = {(cuuint64_t)G.px * sizeof(T), (cuuint64_t)G.plane * sizeof(T)};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
    cuuint32_t es[3] = {1u, 1u, 1u};
    CUresult r = enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                     (void *)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace cspht
