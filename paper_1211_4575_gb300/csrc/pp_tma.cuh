// pp_tma.cuh -- tensor-memory-accelerator (TMA) copies of mesh boxes into
// shared memory, completed on an mbarrier whose wait is bounded in time.
//
// A box of a 3D FP32 mesh array (x fastest) is described by a CUtensorMap that
// the host encodes (cuTensorMapEncodeTiled, reached through the runtime's
// driver entry point, so the library does not link libcuda).  One thread of a
// CTA announces the bytes it expects on the CTA's mbarrier and issues the
// bulk tensor copies; every thread then waits on the barrier's phase.  The
// wait gives up after a time limit: the CTA then records ST_TIMEOUT in the
// status word (PP_ETIMEOUT on the host) and stops, so that no wait can hold
// the GPU.
//
// Rules the callers keep: the innermost box coordinate times 4 bytes is a
// multiple of 16, the array's row and plane strides are multiples of 16 bytes,
// its base is 16-byte aligned, and every box lies inside the array (the host
// checks these before it launches).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp_internal.cuh"

namespace pp {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One arrival per phase (the issuing thread's arrive.expect_tx).
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The issuing thread's arrival, with the bytes the copies of this phase deliver.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// A plain arrival (no bytes): completes a phase that expects none.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase with this parity has completed, for at most limit_ns
// nanoseconds of wall time; false if the limit ran out first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Every thread of the CTA waits for the phase.  True for all of them when it
// completed in time; false for all when any thread's wait ran out: ST_TIMEOUT
// is then set in status and every thread waits once more, again bounded, for
// copies still in flight before the caller stops using the buffer.
__device__ __forceinline__ bool cta_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns, int *status) {
    const bool ok = mbar_wait_bounded(bar, parity, limit_ns);
    if (!__syncthreads_or(!ok)) return true;
    if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    mbar_wait_bounded(bar, parity, limit_ns);
    return false;
}

// Order this CTA's earlier generic-proxy accesses of shared memory before the
// async-proxy writes of copies issued after it (a buffer refilled by TMA).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A tensor map that lives in global memory (written by a host copy before the
// launch) is read through the tensormap proxy: acquire it before use.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

// Copy the box at element coordinates (x, y, z) of the map's array into dst
// (shared, 128-byte aligned); completion is counted on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Host: the tensor map of boxes of box[0] x box[1] x box[2] FP32 elements of a
// dim[0] x dim[1] x dim[2] array (x fastest, rows of dim[0] elements, no gaps)
// at base.  cudaErrorInvalidValue when the layout breaks a TMA rule or the
// encoder is unavailable.
cudaError_t encode_box_map(CUtensorMap *map, const float *base, const int dim[3], const int box[3]);

// Host: one CTA that waits on a staging barrier, bounded by limit_ns, whose
// phase completes (deliver) or never does; a wait that runs out sets
// ST_TIMEOUT in status.
cudaError_t launch_wait_check(cudaStream_t st, int *status, int deliver, uint64_t limit_ns);

}  // namespace pp
