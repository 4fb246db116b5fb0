// pp_tma.cu -- host encoding of the TMA tensor maps, and the check kernel of
// the bounded staging wait.
#include <cudaTypedefs.h>

#include "pp_tma.cuh"

namespace pp {

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (resolved once).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// One CTA: thread 0 opens a phase of the staging barrier and either completes
// it (deliver: a plain arrival) or announces 16 bytes that no copy delivers, so
// that every thread's wait runs out after limit_ns; the result lands in
// status exactly as a staging wait of the particle kernel reports it.
__global__ void k_wait_check(int *status, int deliver, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        if (deliver)
            mbar_arrive(&bar);
        else
            mbar_arrive_expect(&bar, 16);
    }
    __syncthreads();
    cta_wait_bounded(&bar, 0, limit_ns, status);
}

}  // namespace

cudaError_t encode_box_map(CUtensorMap *map, const float *base, const int dim[3], const int box[3]) {
    const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15) != 0 || (dim[0] * sizeof(float)) % 16 != 0 || (box[0] * sizeof(float)) % 16 != 0)
        return cudaErrorInvalidValue;
    for (int a = 0; a < 3; ++a)
        if (box[a] < 1 || box[a] > 256 || box[a] > dim[a]) return cudaErrorInvalidValue;
    const cuuint64_t gdim[3] = {(cuuint64_t)dim[0], (cuuint64_t)dim[1], (cuuint64_t)dim[2]};
    const cuuint64_t gstride[2] = {(cuuint64_t)dim[0] * sizeof(float), (cuuint64_t)dim[0] * dim[1] * sizeof(float)};
    const cuuint32_t bdim[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, gdim, gstride, bdim, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_wait_check(cudaStream_t st, int *status, int deliver, uint64_t limit_ns) {
    k_wait_check<<<1, 128, 0, st>>>(status, deliver, limit_ns);
    return cudaGetLastError();
}

}  // namespace pp
