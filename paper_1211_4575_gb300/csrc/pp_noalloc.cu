// pp_noalloc.cu -- an entry point that allocates nothing: the FP64 field-energy
// reduction of pp_diagnostics, for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc at the point where they
// need the field energies: real-time loops that forbid allocation after
// start-up (an allocation can block or fail at an arbitrary time), or
// embedding hosts that own all device memory and hand the library
// pre-allocated buffers and nothing else.  This variant keeps its scratch (the
// per-block partial sums of the reduction) in a file-scope __device__ array of
// fixed size instead of asking for memory.
//
// The array is one per device that loads the library and lives until the
// process exits.  Host code cannot use the array's name as a device address:
// the first call on a device, with that device current, looks the address up
// with cudaGetSymbolAddress and caches it per device ordinal; make that first
// call before any stream capture.  The cached address belongs to the device's
// context: after cudaDeviceReset it is stale, so a process that resets a
// device must not call this entry point on that device again.  Every call
// shares the array, so calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it.
#include <stdio.h>

#include <mutex>

#include "pp_internal.cuh"

namespace pp {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;            // partial sums per quantity
constexpr int kNaValues = 3;                  // W_E, W_B, W_Ex
constexpr int64_t kNaMaxCells = (int64_t)1023 * 1023 * 1023;

// 1024 blocks x 3 doubles = 24 KiB of scratch per device.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * kNaValues];

struct NaFields {
    const double *E[3];
    const double *B[3];
};

__global__ void __launch_bounds__(kNaThreads) k_na_energy_partials(NaFields f, int64_t cells, double *partials) {
    double v[kNaValues] = {0.0, 0.0, 0.0};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += (int64_t)gridDim.x * blockDim.x) {
        double e0 = f.E[0][t], e1 = f.E[1][t], e2 = f.E[2][t];
        double b0 = f.B[0][t], b1 = f.B[1][t], b2 = f.B[2][t];
        v[0] += e0 * e0 + e1 * e1 + e2 * e2;
        v[1] += b0 * b0 + b1 * b1 + b2 * b2;
        v[2] += e0 * e0;
    }
    __shared__ double sh[kNaValues][kNaThreads];
    for (int m = 0; m < kNaValues; ++m) sh[m][threadIdx.x] = v[m];
    __syncthreads();
    for (int s = kNaThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int m = 0; m < kNaValues; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int m = 0; m < kNaValues; ++m) partials[blockIdx.x * kNaValues + m] = sh[m][0];
}

// One thread per quantity sums the partials in block order (deterministic).
__global__ void k_na_energy_final(const double *partials, int nblk, double scale, double *out) {
    int m = threadIdx.x;
    if (m >= kNaValues) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += partials[b * kNaValues + m];
    out[m] = acc * scale;
}

}  // namespace pp

using namespace pp;

static std::mutex g_na_mutex;
static double *g_na_ptr[64];
static bool g_na_ready[64];

// Device address of this device's partial-sum array (looked up once per device).
static cudaError_t na_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = (double *)p;
        g_na_ready[dev] = true;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

static thread_local char g_na_err[256];

extern "C" const char *pp_field_energy_noalloc_error(void) { return g_na_err; }

extern "C" int pp_field_energy_noalloc(const double *const E[3], const double *const B[3], int nx, int ny, int nz,
                                       double dV, double *out, void *stream) {
    g_na_err[0] = 0;
    if (!E || !B || !out) {
        snprintf(g_na_err, sizeof g_na_err, "pp_field_energy_noalloc: NULL argument");
        return PP_EINVAL;
    }
    for (int a = 0; a < 3; ++a)
        if (!E[a] || !B[a]) {
            snprintf(g_na_err, sizeof g_na_err, "pp_field_energy_noalloc: NULL field component");
            return PP_EINVAL;
        }
    int64_t cells = (int64_t)nx * ny * nz;
    if (nx < 1 || ny < 1 || nz < 1 || cells > kNaMaxCells) {
        snprintf(g_na_err, sizeof g_na_err,
                 "pp_field_energy_noalloc: mesh %d x %d x %d outside 1 .. %lld cells", nx, ny, nz,
                 (long long)kNaMaxCells);
        return PP_EINVAL;
    }
    double *scratch = nullptr;
    cudaError_t e = na_scratch(&scratch);
    if (e != cudaSuccess) {
        snprintf(g_na_err, sizeof g_na_err, "pp_field_energy_noalloc: scratch lookup: %s", cudaGetErrorString(e));
        return PP_ECUDA;
    }
    int64_t want = (cells + kNaThreads - 1) / kNaThreads;
    int nblk = (int)(want < kNaMaxBlocks ? want : kNaMaxBlocks);
    NaFields f{{E[0], E[1], E[2]}, {B[0], B[1], B[2]}};
    cudaStream_t st = (cudaStream_t)stream;
    k_na_energy_partials<<<nblk, kNaThreads, 0, st>>>(f, cells, scratch);
    k_na_energy_final<<<1, 32, 0, st>>>(scratch, nblk, 0.5 * dV, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_na_err, sizeof g_na_err, "pp_field_energy_noalloc: launch: %s", cudaGetErrorString(e));
        return PP_ECUDA;
    }
    return PP_OK;
}
