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
// perm[slot] = particle instead of moving the particles.  The keys sit in the
// last sort's slot order and each particle moved at most a cell, so the keys
// of a block of consecutive slots lie in a short range: each block counts its
// kAggSpan keys in a shared window and reserves one run of slots per distinct
// key with a single global atomic; keys outside the window (a particle that
// left, a far jump) take a global atomic of their own.  The window starts
// kAggMargin keys below the median of the block's first three keys (robust to
// one of them having jumped), which leaves room for particles that moved down
// a cell in z.
constexpr int kAggThreads = 1024;
constexpr int kAggPer = 8;                          // keys per thread
constexpr int kAggSpan = kAggThreads * kAggPer;     // keys per block
constexpr int kAggWindow = 8192;                    // window of keys counted in shared memory
constexpr int kAggMargin = 1024;
static_assert(kAggWindow % kAggThreads == 0, "window must split evenly over the block");
constexpr int32_t kNoKey = 0x7fffffff;

// The kAggPer keys of this thread: two runs of four consecutive slots, each
// one 16-byte load when whole (slot of key 4h + m: base + 4 h kAggThreads + 4 tid + m).
__device__ __forceinline__ void load_keys(const int32_t *keys, int64_t n, int64_t base, int32_t (&k)[kAggPer]) {
#pragma unroll
    for (int h = 0; h < kAggPer / 4; ++h) {
        const int64_t q = base + (int64_t)h * 4 * kAggThreads + 4 * threadIdx.x;
        if (q + 3 < n) {
            const int4 v = __ldg(reinterpret_cast<const int4 *>(keys + q));
            k[4 * h] = v.x;
            k[4 * h + 1] = v.y;
            k[4 * h + 2] = v.z;
            k[4 * h + 3] = v.w;
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) k[4 * h + m] = q + m < n ? keys[q + m] : kNoKey;
        }
    }
}

__device__ __forceinline__ int64_t key_slot(int64_t base, int i) {
    return base + (int64_t)(i >> 2) * 4 * kAggThreads + 4 * threadIdx.x + (i & 3);
}

// First key of the block's window (same value in every thread).
__device__ __forceinline__ int32_t window_start(const int32_t *keys, int64_t n, int64_t base, int32_t *sh) {
    if (threadIdx.x == 0) {
        const int32_t a = keys[base], b = base + 1 < n ? keys[base + 1] : a, c = base + 2 < n ? keys[base + 2] : a;
        const int32_t med = max(min(a, b), min(max(a, b), c));
        sh[0] = med - kAggMargin;
    }
    __syncthreads();
    return sh[0];
}

__global__ void __launch_bounds__(kAggThreads) k_hist(int64_t n, const int32_t *keys, int32_t *counts) {
    __shared__ int32_t cnt[kAggWindow];
    __shared__ int32_t k0s;
    const int64_t base = (int64_t)blockIdx.x * kAggSpan;
    int32_t k[kAggPer];
    load_keys(keys, n, base, k);
    for (int i = threadIdx.x; i < kAggWindow; i += kAggThreads) cnt[i] = 0;
    const int32_t k0 = window_start(keys, n, base, &k0s);
#pragma unroll
    for (int i = 0; i < kAggPer; ++i) {
        if (k[i] == kNoKey) continue;
        const uint32_t r = (uint32_t)k[i] - (uint32_t)k0;
        if (r < (uint32_t)kAggWindow) atomicAdd(cnt + r, 1);
        else atomicAdd(counts + k[i], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kAggWindow; i += kAggThreads)
        if (cnt[i]) atomicAdd(counts + k0 + i, cnt[i]);
}

__global__ void __launch_bounds__(kAggThreads) k_perm(int64_t n, const int32_t *keys, int32_t *cursor, int32_t *perm) {
    __shared__ int32_t cnt[kAggWindow];   // block-local rank counters, then the reserved bases
    __shared__ int32_t k0s;
    const int64_t base = (int64_t)blockIdx.x * kAggSpan;
    int32_t k[kAggPer], rank[kAggPer];
    load_keys(keys, n, base, k);
    for (int i = threadIdx.x; i < kAggWindow; i += kAggThreads) cnt[i] = 0;
    const int32_t k0 = window_start(keys, n, base, &k0s);
#pragma unroll
    for (int i = 0; i < kAggPer; ++i) {
        const uint32_t r = (uint32_t)k[i] - (uint32_t)k0;
        rank[i] = (k[i] != kNoKey && r < (uint32_t)kAggWindow) ? atomicAdd(cnt + r, 1) : -1;
    }
    __syncthreads();
    // one reservation per distinct key; the loop is unrolled so that a
    // thread's atomics (each waits for its returned base) are all in flight
#pragma unroll
    for (int m = 0; m < kAggWindow / kAggThreads; ++m) {
        const int i = threadIdx.x + m * kAggThreads;
        const int32_t c = cnt[i];
        if (c) cnt[i] = atomicAdd(cursor + k0 + i, c);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kAggPer; ++i) {
        if (k[i] == kNoKey) continue;
        const int32_t slot =
            rank[i] >= 0 ? cnt[(uint32_t)k[i] - (uint32_t)k0] + rank[i] : atomicAdd(cursor + k[i], 1);
        perm[slot] = (int32_t)key_slot(base, i);
    }
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
    const unsigned ablocks = (unsigned)((S.n + kAggSpan - 1) / kAggSpan);
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
