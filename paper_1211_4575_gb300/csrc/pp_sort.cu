// pp_sort.cu -- counting sort of a species' particle arrays by cell (Sec. III:
// between the current deposit and the field update the paper sorts the
// particles by their cell, for cache locality).
//
// The key of a particle is its cell, numbered tile by tile (tiles of up to
// 8x8x8 cells, x fastest inside a tile and across tiles), so that the sorted
// arrays hold every tile as one contiguous range, times kSubKeys plus the
// octant of the particle inside its cell (which half of the cell on each
// axis).  The octant order makes particles of equal rank in neighbouring
// cells sit in the same half-cell, so that the lanes of a warp in the tiled
// kernel use the same stencil offsets.  Pipeline: key + histogram
// (warp-aggregated atomics) -> exclusive scan -> scatter through per-key
// cursors.  The order inside a cell is not deterministic.
#include "pp_internal.cuh"

namespace pp {

struct KeyGeom {
    int n[3];
    int T[3];
    int nt[3];
    int64_t tile_vol;
    int32_t dead;   // key of a particle that left the box: after every cell's keys
};

__device__ __forceinline__ int32_t cell_key(const KeyGeom &k, int x, int y, int z) {
    int tx = x / k.T[0], ty = y / k.T[1], tz = z / k.T[2];
    int lx = x - tx * k.T[0], ly = y - ty * k.T[1], lz = z - tz * k.T[2];
    int64_t tile = ((int64_t)tz * k.nt[1] + ty) * k.nt[0] + tx;
    return (int32_t)(tile * k.tile_vol + ((int64_t)lz * k.T[1] + ly) * k.T[0] + lx);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Returns, for every calling lane, a slot from *counter reserved jointly by all
// active lanes with the same key (one atomic per distinct key per warp).
__device__ __forceinline__ int32_t aggregated_add(int32_t *base, int32_t key) {
    unsigned active = __activemask();
    unsigned peers = __match_any_sync(active, key);
    int leader = __ffs(peers) - 1;
    int rank = __popc(peers & lanemask_lt());
    int32_t b = 0;
    if ((int)(threadIdx.x & 31) == leader) b = atomicAdd(base + key, __popc(peers));
    b = __shfl_sync(peers, b, leader);
    return b + rank;
}

__global__ void k_keys_fp64(KeyGeom kg, int64_t n, const double *x, const double *y, const double *z, int32_t *keys,
                            int32_t *counts) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (x[t] < 0.0) {   // left the box
        keys[t] = kg.dead;
        aggregated_add(counts, kg.dead);
        return;
    }
    int cx = (int)floor(x[t]), cy = (int)floor(y[t]), cz = (int)floor(z[t]);
    cx = min(max(cx, 0), kg.n[0] - 1);
    cy = min(max(cy, 0), kg.n[1] - 1);
    cz = min(max(cz, 0), kg.n[2] - 1);
    int oct = (x[t] - cx >= 0.5 ? 1 : 0) | (y[t] - cy >= 0.5 ? 2 : 0) | (z[t] - cz >= 0.5 ? 4 : 0);
    int32_t key = cell_key(kg, cx, cy, cz) * kSubKeys + oct;
    keys[t] = key;
    aggregated_add(counts, key);
}

__global__ void k_keys_mixed(KeyGeom kg, int64_t n, const int32_t *cell, const float *ox, const float *oy,
                             const float *oz, int32_t *keys, int32_t *counts) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t c = cell[t];
    if (c < 0) {   // left the box
        keys[t] = kg.dead;
        aggregated_add(counts, kg.dead);
        return;
    }
    int oct = (ox[t] >= 0.5f ? 1 : 0) | (oy[t] >= 0.5f ? 2 : 0) | (oz[t] >= 0.5f ? 4 : 0);
    int32_t key = cell_key(kg, c & 1023, (c >> 10) & 1023, (c >> 20) & 1023) * kSubKeys + oct;
    keys[t] = key;
    aggregated_add(counts, key);
}

// ---- exclusive scan of int32 counts (multi-level, 2048 values per block) ----
constexpr int kScanThreads = 256, kScanPer = 8, kScanChunk = kScanThreads * kScanPer;

__global__ void k_scan_block(const int32_t *in, int32_t *out, int64_t n, int32_t *sums) {
    __shared__ int32_t sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
    int32_t v[kScanPer];
    int32_t local = 0;
#pragma unroll
    for (int m = 0; m < kScanPer; ++m) {
        int64_t q = base + m;
        v[m] = q < n ? in[q] : 0;
        local += v[m];
    }
    sh[threadIdx.x] = local;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        int32_t a = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += a;
        __syncthreads();
    }
    int32_t run = sh[threadIdx.x] - local;   // exclusive prefix of this thread
#pragma unroll
    for (int m = 0; m < kScanPer; ++m) {
        int64_t q = base + m;
        if (q < n) out[q] = run;
        run += v[m];
    }
    if (threadIdx.x == kScanThreads - 1 && sums) sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *sums) {
    int64_t q = (int64_t)blockIdx.x * kScanChunk + threadIdx.x;
    int32_t add = sums[blockIdx.x];
    for (int m = 0; m < kScanPer; ++m, q += kScanThreads)
        if (q < n) out[q] += add;
}

// tmp must hold the block sums of every level (sum of ceil(n / 2048^l)).
static cudaError_t scan(cudaStream_t st, const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, int64_t &nl) {
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb <= 1) {
        k_scan_block<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        ++nl;
        return cudaGetLastError();
    }
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, tmp);
    ++nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan(st, tmp, tmp, nb, tmp + nb, nl);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, tmp);
    ++nl;
    return cudaGetLastError();
}

static size_t scan_tmp_count(int64_t n) {
    size_t total = 0;
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    while (nb > 1) {
        total += (size_t)nb;
        nb = (nb + kScanChunk - 1) / kScanChunk;
    }
    return total + 1;
}

template <typename T>
__device__ __forceinline__ void mv(const T *src, T *dst, int64_t from, int64_t to) {
    dst[to] = src[from];
}

__global__ void k_scatter_fp64(int64_t n, const int32_t *keys, int32_t *cursor, const double *x, const double *y,
                               const double *z, const double *ux, const double *uy, const double *uz, double *x2,
                               double *y2, double *z2, double *ux2, double *uy2, double *uz2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t p = aggregated_add(cursor, keys[t]);
    mv(x, x2, t, p); mv(y, y2, t, p); mv(z, z2, t, p);
    mv(ux, ux2, t, p); mv(uy, uy2, t, p); mv(uz, uz2, t, p);
}

__global__ void k_scatter_mixed(int64_t n, const int32_t *keys, int32_t *cursor, const int32_t *cell, const float *ox,
                                const float *oy, const float *oz, const float *ux, const float *uy, const float *uz,
                                int32_t *cell2, float *ox2, float *oy2, float *oz2, float *ux2, float *uy2,
                                float *uz2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t p = aggregated_add(cursor, keys[t]);
    mv(cell, cell2, t, p);
    mv(ox, ox2, t, p); mv(oy, oy2, t, p); mv(oz, oz2, t, p);
    mv(ux, ux2, t, p); mv(uy, uy2, t, p); mv(uz, uz2, t, p);
}

// Sort from keys a particle pass already wrote (Species::keys_valid): the
// histogram of the keys, then, through the per-key cursors, the permutation
// perm[slot] = particle instead of moving the particles.  The keys of a block
// of consecutive particles (in the last sort's order) lie in a short range, so
// each block counts its keys in shared memory and reserves one run of slots
// per distinct key with a single global atomic; keys outside the block's
// window (a particle that left, a far jump) take a global atomic of their own.
constexpr int kAggThreads = 1024;
constexpr int kAggWindow = 4096;   // keys counted in shared memory per block

__device__ __forceinline__ int32_t block_min_key(int32_t k, int32_t *sh) {
    // smallest live key of the block (keys >= sentinel are ignored)
    int32_t v = k;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t w = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = min(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) sh[32] = w;
    }
    __syncthreads();
    return sh[32];
}

__global__ void __launch_bounds__(kAggThreads) k_hist(int64_t n, const int32_t *keys, int32_t *counts) {
    __shared__ int32_t cnt[kAggWindow];
    __shared__ int32_t red[33];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t key = t < n ? keys[t] : 0x7fffffff;
    const int32_t k0 = block_min_key(key, red);
    for (int i = threadIdx.x; i < kAggWindow; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    if (t < n) {
        const int32_t r = key - k0;
        if (r < kAggWindow) atomicAdd(cnt + r, 1);
        else atomicAdd(counts + key, 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kAggWindow; i += blockDim.x)
        if (cnt[i]) atomicAdd(counts + k0 + i, cnt[i]);
}

__global__ void __launch_bounds__(kAggThreads) k_perm(int64_t n, const int32_t *keys, int32_t *cursor, int32_t *perm) {
    __shared__ int32_t cnt[kAggWindow];   // block-local rank counters, then the reserved bases
    __shared__ int32_t red[33];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t key = t < n ? keys[t] : 0x7fffffff;
    const int32_t k0 = block_min_key(key, red);
    for (int i = threadIdx.x; i < kAggWindow; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int32_t r = key - k0;
    const bool local = t < n && r < kAggWindow;
    int32_t rank = 0;
    if (local) rank = atomicAdd(cnt + r, 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kAggWindow; i += blockDim.x)
        if (cnt[i]) cnt[i] = atomicAdd(cursor + k0 + i, cnt[i]);
    __syncthreads();
    if (local) perm[cnt[r] + rank] = (int32_t)t;
    else if (t < n) perm[atomicAdd(cursor + key, 1)] = (int32_t)t;
}

// dst[i] = src[perm[i]] for the seven arrays of the mixed form.
__global__ void k_apply_perm(int64_t n, const int32_t *perm, const int32_t *cell, const float *ox, const float *oy,
                             const float *oz, const float *ux, const float *uy, const float *uz, int32_t *cell2,
                             float *ox2, float *oy2, float *oz2, float *ux2, float *uy2, float *uz2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t t = perm[i];
    mv(cell, cell2, t, i);
    mv(ox, ox2, t, i); mv(oy, oy2, t, i); mv(oz, oz2, t, i);
    mv(ux, ux2, t, i); mv(uy, uy2, t, i); mv(uz, uz2, t, i);
}

static void swap_buffers(Ctx &c, Species &S) {
    void *old = S.buf;
    S.buf = S.alt;
    S.alt = old;
    S.bind(c.fp64);
}

cudaError_t materialize(Ctx &c, int s) {
    Species &S = c.sp[s];
    if (!S.perm_pending) return cudaSuccess;
    S.perm_pending = false;
    if (S.n == 0) return cudaSuccess;
    const int64_t cp = S.cap;
    int32_t *c2 = (int32_t *)S.alt;
    float *f2 = (float *)(c2 + cp);
    k_apply_perm<<<(unsigned)((S.n + 255) / 256), 256, 0, c.st>>>(S.n, S.perm, S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy,
                                                                 S.fuz, c2, f2, f2 + cp, f2 + 2 * cp, f2 + 3 * cp,
                                                                 f2 + 4 * cp, f2 + 5 * cp);
    ++c.nlaunch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    swap_buffers(c, S);
    return cudaSuccess;
}

static KeyGeom key_geom(const Ctx &c) {
    KeyGeom k;
    for (int a = 0; a < 3; ++a) {
        k.n[a] = c.g.n[a];
        k.T[a] = c.tile[a];
        k.nt[a] = c.ntile[a];
    }
    k.tile_vol = (int64_t)c.tile[0] * c.tile[1] * c.tile[2];
    k.dead = (int32_t)c.nkeys;
    return k;
}

cudaError_t sort_setup(Ctx &c) {
    for (int a = 0; a < 3; ++a) {
        c.tile[a] = c.g.n[a] < 8 ? c.g.n[a] : 8;
        c.ntile[a] = (c.g.n[a] + c.tile[a] - 1) / c.tile[a];
    }
    c.nkeys = (int64_t)c.ntile[0] * c.ntile[1] * c.ntile[2] * c.tile[0] * c.tile[1] * c.tile[2] * kSubKeys;
    cudaError_t e = cudaMalloc(&c.counts, sizeof(int32_t) * (c.nkeys + 1));
    if (e != cudaSuccess) return e;
    c.scan_tmp_bytes = sizeof(int32_t) * scan_tmp_count(c.nkeys + 1);
    return cudaMalloc(&c.scan_tmp, c.scan_tmp_bytes);
}

// Particles that left the box sort after every cell (key nkeys); when the
// species may hold some, the live count cell_start[nkeys] is read back (a
// synchronisation) and becomes the species' count, which drops them.
cudaError_t launch_sort(Ctx &c, int s) {
    Species &S = c.sp[s];
    S.sorted = true;
    // keys from the last particle pass: no key pass, and a permutation in
    // place of the scatter; otherwise the arrays are put in order first
    const bool lazy = S.keys_valid && !S.perm_pending && !c.fp64 && S.n > 0;
    S.keys_valid = false;
    cudaError_t e = lazy ? cudaSuccess : materialize(c, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c.counts, 0, sizeof(int32_t) * (c.nkeys + 1), c.st);
    if (e != cudaSuccess) return e;
    if (S.n == 0) {
        S.nsorted = 0;
        S.may_hold_dead = false;
        S.fresh = true;
        return cudaMemsetAsync(S.cell_start, 0, sizeof(int32_t) * (c.nkeys + 1), c.st);
    }
    KeyGeom kg = key_geom(c);
    unsigned blocks = (unsigned)((S.n + 255) / 256);
    const unsigned ablocks = (unsigned)((S.n + kAggThreads - 1) / kAggThreads);
    if (lazy) k_hist<<<ablocks, kAggThreads, 0, c.st>>>(S.n, S.keys, c.counts);
    else if (c.fp64) k_keys_fp64<<<blocks, 256, 0, c.st>>>(kg, S.n, S.x, S.y, S.z, S.keys, c.counts);
    else k_keys_mixed<<<blocks, 256, 0, c.st>>>(kg, S.n, S.cell, S.ox, S.oy, S.oz, S.keys, c.counts);
    ++c.nlaunch;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // cell_start = exclusive scan of counts; counts then becomes the cursor
    if ((e = scan(c.st, c.counts, S.cell_start, c.nkeys + 1, (int32_t *)c.scan_tmp, c.nlaunch)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(c.counts, S.cell_start, sizeof(int32_t) * (c.nkeys + 1), cudaMemcpyDeviceToDevice, c.st);
    if (e != cudaSuccess) return e;
    if (lazy) {
        k_perm<<<ablocks, kAggThreads, 0, c.st>>>(S.n, S.keys, c.counts, S.perm);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        S.perm_pending = true;
    } else if (c.fp64) {
        double *b = (double *)S.alt;
        int64_t cp = S.cap;
        k_scatter_fp64<<<blocks, 256, 0, c.st>>>(S.n, S.keys, c.counts, S.x, S.y, S.z, S.ux, S.uy, S.uz, b, b + cp,
                                                 b + 2 * cp, b + 3 * cp, b + 4 * cp, b + 5 * cp);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        void *old = S.buf;
        S.buf = S.alt;
        S.alt = old;
        S.bind(true);
    } else {
        int64_t cp = S.cap;
        int32_t *c2 = (int32_t *)S.alt;
        float *f2 = (float *)(c2 + cp);
        k_scatter_mixed<<<blocks, 256, 0, c.st>>>(S.n, S.keys, c.counts, S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz,
                                                  c2, f2, f2 + cp, f2 + 2 * cp, f2 + 3 * cp, f2 + 4 * cp, f2 + 5 * cp);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        void *old = S.buf;
        S.buf = S.alt;
        S.alt = old;
        S.bind(false);
    }
    if (S.may_hold_dead) {
        e = cudaMemcpyAsync(c.h_count, S.cell_start + c.nkeys, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) return e;
        S.n = *c.h_count;
        S.may_hold_dead = false;
    }
    S.nsorted = S.n;
    S.fresh = true;
    return cudaSuccess;
}

}  // namespace pp
