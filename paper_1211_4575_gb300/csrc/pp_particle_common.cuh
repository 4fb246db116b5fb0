// pp_particle_common.cuh -- per-particle helpers shared by the particle
// kernels (pp_particles.cu, pp_cells.cu): the two particle layouts, the packed
// cell of the mixed form, the re-binning of a moved offset and the reflection
// at walls (Sec. V "Boundary conditions").
#pragma once

#include "pp_internal.cuh"

namespace pp {

struct Fp64Particles {
    double *x, *y, *z, *ux, *uy, *uz;
};

struct MixedParticles {
    int32_t *cell;
    float *ox, *oy, *oz, *ux, *uy, *uz;
};

__device__ __forceinline__ void unpack_cell(int32_t c, int &x, int &y, int &z) {
    x = c & 1023;
    y = (c >> 10) & 1023;
    z = (c >> 20) & 1023;
}
__device__ __forceinline__ int32_t pack_cell(int x, int y, int z) { return x | (y << 10) | (z << 20); }

// Re-bin an offset that moved by less than one cell: offset back into [0,1),
// cell index shifted and wrapped.  An offset that rounds to exactly 1 after
// adding 1 belongs to the cell above with offset 0.
__device__ __forceinline__ void rebin(float &o, int &c, int n) {
    if (o >= 1.0f) {
        o -= 1.0f;
        ++c;
    } else if (o < 0.0f) {
        o += 1.0f;
        --c;
        if (o >= 1.0f) {
            o = 0.0f;
            ++c;
        }
    }
    if (c < 0) c += n;
    else if (c >= n) c -= n;
}

// Reflecting walls at 0 and nw cells on one axis (Sec. V "Boundary
// conditions"), applied after the particle deposited its step as if streaming
// freely: a particle that ended the move beyond a wall (in (nw, 2 nw) of the
// mirror-extended box, which the periodic wrap also gives below 0) is replaced
// by its virtual image, x -> 2 nw - x and u -> -u along that axis.  nw = 0: no
// walls on the axis.
__device__ __forceinline__ void reflect(double &xi, double &ux, int nw) {
    if (nw && xi > (double)nw) {
        xi = 2.0 * (double)nw - xi;
        ux = -ux;
    }
}
// Mixed form: cell cx and offset o in [0, 1).  2 nw - (cx + o) is cell
// 2 nw - 1 - cx with offset 1 - o, or cell 2 nw - cx when o = 0; an offset
// that rounds to 1 moves to the cell above.
__device__ __forceinline__ void reflect(int &cx, float &o, float &ux, int nw) {
    if (nw && (cx > nw || (cx == nw && o > 0.0f))) {
        if (o > 0.0f) {
            cx = 2 * nw - 1 - cx;
            o = 1.0f - o;
            if (o >= 1.0f) {
                o = 0.0f;
                ++cx;
            }
        } else {
            cx = 2 * nw - cx;
        }
        ux = -ux;
    }
}

// The opt-in dynamic shared memory of a kernel, set once per device (the
// attribute belongs to the device's context; a bit per device ordinal).  Two
// threads that race here set the same value.
template <class K>
static cudaError_t ensure_smem_attr(K kernel, int bytes, unsigned long long &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}

}  // namespace pp
