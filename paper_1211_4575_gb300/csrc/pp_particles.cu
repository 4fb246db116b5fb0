// pp_particles.cu -- per-particle kernels: the fused gather -> push -> move ->
// charge-conserving deposit (Sec. III steps 1-3) in its one-thread-per-particle
// form, the charge density of eq:rho2, the kinetic-energy reduction and the
// FP64 <-> storage conversions of pp_load_particles / pp_get_particles.
#include "pp_internal.cuh"
#include "pp_particle_common.cuh"

namespace pp {

// Frame accessor over the padded global mesh: frame index (i,j,k) means mesh
// index (ox+i, oy+j, oz+k).  Fields read through the read-only path, current
// accumulated with device-scope atomics.
template <typename R>
struct GlobalAcc {
    Geom g;
    const R *E[3];
    const R *B[3];
    R *J[3];
    int ox, oy, oz;
    PP_IF_CHECKED(int *st = nullptr; mutable int bad = 0;)
#ifdef PP_CHECKED
    __device__ __forceinline__ bool inside(int x, int y, int z) const {
        return x >= -g.G && x < g.n[0] + g.G && y >= -g.G && y < g.n[1] + g.G && z >= -g.G && z < g.n[2] + g.G;
    }
    __device__ ~GlobalAcc() {   // one report per particle
        if (bad && st) atomicOr(st, ST_BOUNDS);
    }
#endif
    __device__ __forceinline__ R F(int kind, int comp, int i, int j, int k) const {
        PP_IF_CHECKED(if (!inside(ox + i, oy + j, oz + k)) { bad = 1; return R(0); })
        const R *p = kind ? B[comp] : E[comp];
        return __ldg(p + g.at(ox + i, oy + j, oz + k));
    }
    __device__ __forceinline__ void addJ(int comp, int i, int j, int k, R v) const {
        PP_IF_CHECKED(if (!inside(ox + i, oy + j, oz + k)) { bad = 1; return; })
        atomicAdd(J[comp] + g.at(ox + i, oy + j, oz + k), v);
    }
};

template <typename R>
struct StepArgs {
    Geom g;
    const R *E[3];
    const R *B[3];
    R *J[3];
    R qmdt;
    R kdt;                       // radiative cooling K / dt (0 = off)
    R dtdx[3];
    R jscale[3];
    int64_t n;
    int *status;
    int direct;                  // 1: direct current eq:jj2; 0: charge-conserving
    int wall[3];                 // walls at 0 and wall[a] cells on axis a; 0 = periodic
    double esc;                  // open end: outgoing particles below x = esc cells leave; 0 = off
    int64_t off;                 // first particle of the launch
};

template <int O, int PUSH>
__global__ void __launch_bounds__(256) k_particles_fp64(StepArgs<double> a, Fp64Particles p) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    t += a.off;
    if (p.x[t] < 0.0) return;   // left the box
    double xi0[3] = {p.x[t], p.y[t], p.z[t]};
    double u[3] = {p.ux[t], p.uy[t], p.uz[t]};
    GlobalAcc<double> acc{a.g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, 0, 0, 0};
    PP_IF_CHECKED(acc.st = a.status;)
    if (a.qmdt != 0.0) {   // no kick (a 4th-order drift-only substep, or q = 0): no force
        double E[3], B[3];
        gather_EB<O, double>(acc, xi0, E, B);
        push_particle<PUSH, double>(a.qmdt, a.kdt, E, B, u);
    }
    double gi = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double xi1[3], dxs[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double dx = a.dtdx[d] * u[d] * gi;
        dxs[d] = dx;
        xi1[d] = xi0[d] + dx;
        ok = ok && (fabs(dx) < 1.0);   // also false for NaN
    }
    if (!ok) {
        atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
        return;
    }
    if (a.direct) deposit_direct<O, double>(acc, xi0, dxs, a.jscale);
    else deposit_esirkepov<O, double>(acc, xi0, xi1, a.jscale);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double L = (double)a.g.n[d], v = xi1[d];
        if (v < 0.0) v += L;
        else if (v >= L) v -= L;
        if (v >= L) v -= L;
        xi1[d] = v;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) reflect(xi1[d], u[d], a.wall[d]);
    if (a.esc > 0.0 && xi1[0] < a.esc && u[0] < 0.0) xi1[0] = kDeadX;   // out through the open end
    p.x[t] = xi1[0]; p.y[t] = xi1[1]; p.z[t] = xi1[2];
    p.ux[t] = u[0]; p.uy[t] = u[1]; p.uz[t] = u[2];
}

template <int O, int PUSH>
__global__ void __launch_bounds__(256) k_particles_mixed(StepArgs<float> a, MixedParticles p) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    t += a.off;
    if (p.cell[t] < 0) return;   // left the box
    int cx, cy, cz;
    unpack_cell(p.cell[t], cx, cy, cz);
    float xi0[3] = {p.ox[t], p.oy[t], p.oz[t]};
    float u[3] = {p.ux[t], p.uy[t], p.uz[t]};
    GlobalAcc<float> acc{a.g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, cx, cy, cz};
    PP_IF_CHECKED(acc.st = a.status;)
    if (a.qmdt != 0.0f) {   // no kick (a 4th-order drift-only substep, or q = 0): no force
        float E[3], B[3];
        gather_EB<O, float>(acc, xi0, E, B);
        push_particle<PUSH, float>(a.qmdt, a.kdt, E, B, u);
    }
    float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    float xi1[3], dxs[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float dx = a.dtdx[d] * u[d] * gi;
        dxs[d] = dx;
        xi1[d] = xi0[d] + dx;
        ok = ok && (fabsf(dx) < 1.0f);
    }
    if (!ok) {
        atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
        return;
    }
    if (a.direct) deposit_direct<O, float>(acc, xi0, dxs, a.jscale);
    else deposit_esirkepov<O, float>(acc, xi0, xi1, a.jscale);
    rebin(xi1[0], cx, a.g.n[0]);
    rebin(xi1[1], cy, a.g.n[1]);
    rebin(xi1[2], cz, a.g.n[2]);
    reflect(cx, xi1[0], u[0], a.wall[0]);
    reflect(cy, xi1[1], u[1], a.wall[1]);
    reflect(cz, xi1[2], u[2], a.wall[2]);
    int32_t cw = pack_cell(cx, cy, cz);
    if (a.esc > 0.0 && (double)cx + (double)xi1[0] < a.esc && u[0] < 0.0f) cw |= kDeadBit;
    p.cell[t] = cw;
    p.ox[t] = xi1[0]; p.oy[t] = xi1[1]; p.oz[t] = xi1[2];
    p.ux[t] = u[0]; p.uy[t] = u[1]; p.uz[t] = u[2];
}

template <typename R>
static StepArgs<R> step_args(Ctx &c, int s) {
    StepArgs<R> a;
    a.g = c.g;
    for (int d = 0; d < 3; ++d) {
        a.E[d] = (const R *)c.E[d];
        a.B[d] = (const R *)c.B[d];
        a.J[d] = (R *)c.J[d];
    }
    const Species &S = c.sp[s];
    double h[3] = {c.d.dx, c.d.dy, c.d.dz};
    a.qmdt = (R)(S.q * c.kick_dt / S.m);
    a.kdt = (R)(c.kick_dt != 0.0 ? S.rad / c.kick_dt : 0.0);
    for (int d = 0; d < 3; ++d) {
        a.dtdx[d] = (R)(c.drift_dt / h[d]);
        a.jscale[d] = (R)(-S.q * S.w * h[d] / c.drift_dt);
    }
    a.n = S.n;
    a.status = c.d_status;
    a.direct = c.current_mode == PP_CURRENT_DIRECT ? 1 : 0;
    for (int d = 0; d < 3; ++d) a.wall[d] = c.wall[d];
    a.esc = c.escape_now;
    a.off = 0;
    return a;
}

cudaError_t launch_particles_fp64(Ctx &c, int s) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    StepArgs<double> a = step_args<double>(c, s);
    Fp64Particles p{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    unsigned blocks = (unsigned)((S.n + 255) / 256);
    int o = c.d.shape_order, pu = c.d.pusher;
#define PP_L(O, PU) k_particles_fp64<O, PU><<<blocks, 256, 0, c.st>>>(a, p)
    if (pu == PP_BORIS) {
        if (o == 1) PP_L(1, PP_BORIS); else if (o == 2) PP_L(2, PP_BORIS); else PP_L(3, PP_BORIS);
    } else {
        if (o == 1) PP_L(1, PP_VAY); else if (o == 2) PP_L(2, PP_VAY); else PP_L(3, PP_VAY);
    }
#undef PP_L
    ++c.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_particles_mixed_global(Ctx &c, int s) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    S.keys_valid = false;
    StepArgs<float> a = step_args<float>(c, s);
    MixedParticles p{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    unsigned blocks = (unsigned)((S.n + 255) / 256);
    int o = c.d.shape_order, pu = c.d.pusher;
#define PP_L(O, PU) k_particles_mixed<O, PU><<<blocks, 256, 0, c.st>>>(a, p)
    if (pu == PP_BORIS) {
        if (o == 1) PP_L(1, PP_BORIS); else if (o == 2) PP_L(2, PP_BORIS); else PP_L(3, PP_BORIS);
    } else {
        if (o == 1) PP_L(1, PP_VAY); else if (o == 2) PP_L(2, PP_VAY); else PP_L(3, PP_VAY);
    }
#undef PP_L
    ++c.nlaunch;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tiled form (mixed precision).  One CTA per 8x8x8 cell tile of the last cell
// sort, all species in one launch.  The E/B nodes the tile's particles can
// touch are staged in shared memory, and the current is accumulated in a shared
// int32 fixed-point window (native shared integer atomics; FP32 shared
// atomics are several times slower on this part) that each chunk of
// particles flushes, over the box it touched, into the FP32 global mesh.
//
// Fixed point, chosen per chunk and per current component a: the chunk is
// first gathered, pushed and moved; then, with |C Y| <= K_O |dxi_a|
// (fixed_point_cy_bound: K_3 = 1/3 for PCS), no node can receive more than
//     bound_a = K_O |jscale_a| sum_p (|dxi_{p,a}| + 1e-6)
// (the 1e-6 per particle covers the FP32 rounding of the weights in C)
// from the chunk, and the unit 2^30 / bound_a keeps every int32 sum below
// 2^30 (plus at most 1024 rounding halves).  The rounding of a contribution
// is half a unit, i.e. relative to the chunk's total motion rather than to
// the largest possible current; the sum inside a chunk is exact and does not
// depend on the order of the atomics.
//
// A particle may have drifted since the sort: it is handled from shared
// memory while its cell lies within kMargin cells of the tile (minimal
// periodic image); otherwise its index is appended to a per-species list and
// k_particles_listed advances it through the global mesh afterwards (counted
// in n_slow).
// ---------------------------------------------------------------------------
constexpr int kTile = 8;                       // tile edge (cells)
constexpr int kTileCells = kTile * kTile * kTile;
// 1024 threads: 32 warps per SM (one CTA fits, by shared memory) at 64
// registers a thread with no spills; the kernel waits on shared-memory latency,
// and twice the warps of a 512-thread CTA hide more of it (64^3 thermal PCS:
// 3.53 -> 3.39 ms; the Weibel variant, with more queued deposits: 4.10 -> 3.77 ms).
#ifndef PP_TILED_THREADS
#define PP_TILED_THREADS 1024
#endif
constexpr int kThreads = PP_TILED_THREADS;     // threads per tile CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMargin = 2;                     // drift allowed before the fallback
constexpr int kReachLo = 2, kReachHi = 3;      // deposit/gather reach around a cell
constexpr int kWin = kTile + 2 * kMargin + kReachLo + kReachHi;   // 17 nodes per axis
// Window layout: x fastest, then z (stride kWin), then y (stride kWinPlane).
// A warp's lanes take particles about one cell apart in sorted order (lane_q),
// i.e. one per cell over an 8 x 4 block of cells in x and y.  With y strided by a plane of
// 296 = 8 (mod 32) words those 32 cells start in 32 distinct banks; a plain
// 17 x 17 plane folds the block's rows onto each other (2-way conflicts).
constexpr int kWinPlane = 296;
static_assert(kWinPlane >= kWin * kWin && kWinPlane % 32 == 8, "plane pitch must hold a 17 x 17 plane, 8 mod 32");
constexpr int kWinVol = kWinPlane * kWin;      // words per window component
__device__ __forceinline__ int win(int i, int j, int k) { return j * kWinPlane + k * kWin + i; }
constexpr int kWinLo = kMargin + kReachLo;     // window node 0 = tile origin - kWinLo
constexpr int kChunk = 1024;                   // particles staged per round
constexpr int kPerThread = kChunk / kThreads;  // particles per thread per round
constexpr int kRounds = kChunk / 32;           // warp-rounds per chunk
static_assert(kChunk % kThreads == 0 && kRounds == kWarps * kPerThread, "chunk must split evenly over the CTA");
constexpr int kStage = kChunk + kChunk / 32;   // one pad word per 32 (bank spread)
constexpr int kStageArrays = 10;               // cell, 3 offsets, 3 momenta, 3 displacements
constexpr size_t kTiledSmem = sizeof(float) * (9 * kWinVol + kStageArrays * kStage) + sizeof(int) * (16 + kChunk);
static_assert(kTiledSmem <= 227 * 1024, "tile CTA must fit the opt-in shared memory");
constexpr float kFixedRange = 1073741824.0f;   // 2^30
constexpr int32_t kQueued = 1 << 30;           // staging flag on a packed cell (bits 0-29 hold x, y, z)
static_assert(kWarps >= 3, "the queue pass needs three warps per group");
static_assert(kChunk <= 1024, "the fixed-point bound allows at most 1024 rounding halves per flush");
constexpr int kMaxTiledSpecies = PP_MAX_SPECIES;

// Chunk position of the particle that `lane` takes in warp-round j (0..31):
// lanes 2^sh apart in sorted order, j choosing the offset inside that stride
// and the block of 32 * 2^sh particles.  With 2^sh about the number of
// particles per cell, the lanes of a warp sit in 32 consecutive cells.  A
// bijection of (lane, j) onto 0..1023 for sh in 0..5.
__device__ __forceinline__ int lane_q(int lane, int j, int sh) {
    return ((j >> sh) << (sh + 5)) + (lane << sh) + (j & ((1 << sh) - 1));
}

struct SmemAcc {
    const float *Fw;  // 6 windows: E0 E1 E2 B0 B1 B2
    int *J;           // 3 fixed-point windows
    int base;         // window offset of the particle's cell
    PP_IF_CHECKED(int wx = 0, wy = 0, wz = 0; int *st = nullptr; mutable int bad = 0;)   // its window coordinates
#ifdef PP_CHECKED
    __device__ __forceinline__ bool inside(int i, int j, int k) const {
        return wx + i >= 0 && wx + i < kWin && wy + j >= 0 && wy + j < kWin && wz + k >= 0 && wz + k < kWin;
    }
    __device__ ~SmemAcc() {   // one report per particle
        if (bad && st) atomicOr(st, ST_BOUNDS);
    }
#endif
    __device__ __forceinline__ int at(int i, int j, int k) const { return base + win(i, j, k); }
    __device__ __forceinline__ float F(int kind, int comp, int i, int j, int k) const {
        PP_IF_CHECKED(if (!inside(i, j, k)) { bad = 1; return 0.0f; })
        return Fw[(kind * 3 + comp) * kWinVol + at(i, j, k)];
    }
    // v is pre-scaled by the fixed-point unit.  Zero contributions are added
    // too: a per-site test costs more than the extra shared-memory traffic.
    __device__ __forceinline__ void addJ(int comp, int i, int j, int k, float v) const {
        PP_IF_CHECKED(if (!inside(i, j, k)) { bad = 1; return; })
        atomicAdd(J + comp * kWinVol + at(i, j, k), __float2int_rn(v));
    }
};

struct TiledSpecies {
    MixedParticles p;
    const int32_t *cell_start;   // per sort key, tile-major
    int32_t *slow_list;          // indices of particles left to the global-mesh kernel
    unsigned *slow_count;
    float qmdt;
    float kdt;                   // radiative cooling K / dt (0 = off)
    float jscale[3];             // -q w dx_a / dt
    int lane_shift;              // log2 of the sorted-order distance between lanes
};

struct TiledArgs {
    Geom g;
    const float *E[3];
    const float *B[3];
    float *J[3];
    float dtdx[3];
    int nt[3];                   // tiles per axis
    int ns;
    TiledSpecies sp[kMaxTiledSpecies];
    int *status;
    int direct;                  // 1: direct current eq:jj2; 0: charge-conserving
    int wall[3];                 // walls at 0 and wall[a] cells on axis a; 0 = periodic
    double esc;                  // open end: outgoing particles below x = esc cells leave; 0 = off
};

__device__ __forceinline__ int min_image(int d, int n) {
    if (d > n / 2) d -= n;
    else if (d < -(n / 2)) d += n;
    return d;
}

// BND: walls (reflection) and particles that leave (skip, escape); a separate
// instantiation so that periodic runs carry none of their tests.
template <int O, int PUSH, bool BND>
__global__ void __launch_bounds__(kThreads, 1) k_particles_tiled(const __grid_constant__ TiledArgs T) {
    extern __shared__ float smem[];
    float *F = smem;
    int *Jw = (int *)(smem + 6 * kWinVol);
    float *stg = smem + 9 * kWinVol;
    int32_t *s_cell = (int32_t *)stg;
    float *s_o = stg + kStage;           // 3 arrays: offsets at t
    float *s_u = stg + 4 * kStage;       // 3 arrays: momenta
    float *s_d = stg + 7 * kStage;       // 3 arrays: displacement of the step (NaN: not deposited here)
    int *bbox = (int *)(stg + kStageArrays * kStage);   // min x,y,z, max x,y,z of the deposited cells
    int *nqueue = bbox + 6;                               // particles queued for the general deposit
    float *tot = (float *)(bbox + 8);                     // sum |dxi| per axis
    int *s_queue = bbox + 16;                             // their staging indices (kChunk)
    const Geom &g = T.g;
    const int tile = blockIdx.x;
    const int tx = tile % T.nt[0], ty = (tile / T.nt[0]) % T.nt[1], tz = tile / (T.nt[0] * T.nt[1]);
    const int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
    const int wx = ox - kWinLo, wy = oy - kWinLo, wz = oz - kWinLo;
    {   // a tile that holds no particle (the mirror half of a box between walls) stages nothing
        int held = 0;
        for (int s = 0; s < T.ns; ++s)
            held |= T.sp[s].cell_start[(tile + 1) * kTileCells * kSubKeys] - T.sp[s].cell_start[tile * kTileCells * kSubKeys];
        if (!held) return;
    }
    // stage E and B (ghost layers hold the periodic images), clear the current window
    for (int idx = threadIdx.x; idx < 6 * kWinVol; idx += kThreads) {
        int comp = idx / kWinVol, r = idx - comp * kWinVol;
        int j = r / kWinPlane, rem = r - j * kWinPlane;
        if (rem >= kWin * kWin) continue;   // plane padding, never read
        int i = rem % kWin, k = rem / kWin;
        const float *src = comp < 3 ? T.E[comp] : T.B[comp - 3];
#ifdef PP_CHECKED
        if (wx + i < -g.G || wx + i >= g.n[0] + g.G || wy + j < -g.G || wy + j >= g.n[1] + g.G || wz + k < -g.G ||
            wz + k >= g.n[2] + g.G) {
            atomicOr(T.status, ST_BOUNDS);
            F[idx] = 0.0f;
            continue;
        }
#endif
        F[idx] = __ldg(src + g.at(wx + i, wy + j, wz + k));
    }
    for (int idx = threadIdx.x; idx < 3 * kWinVol; idx += kThreads) Jw[idx] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < T.ns; ++s) {
        const TiledSpecies &S = T.sp[s];
        const int tb = S.cell_start[tile * kTileCells * kSubKeys], te = S.cell_start[(tile + 1) * kTileCells * kSubKeys];
        for (int cb = tb; cb < te; cb += kChunk) {
            const int cn = min(kChunk, te - cb);
            if (threadIdx.x < 3) {
                bbox[threadIdx.x] = 1 << 20;          // running minimum
                bbox[3 + threadIdx.x] = -(1 << 20);   // running maximum
                tot[threadIdx.x] = 0.0f;
            }
            if (threadIdx.x == 0) *nqueue = 0;
            for (int q = threadIdx.x; q < cn; q += kThreads) {
                int sq = q + (q >> 5);
                s_cell[sq] = S.p.cell[cb + q];
                s_o[sq] = S.p.ox[cb + q]; s_o[kStage + sq] = S.p.oy[cb + q]; s_o[2 * kStage + sq] = S.p.oz[cb + q];
                s_u[sq] = S.p.ux[cb + q]; s_u[kStage + sq] = S.p.uy[cb + q]; s_u[2 * kStage + sq] = S.p.uz[cb + q];
            }
            __syncthreads();
            // ---- phase 1: gather, push, move (displacements kept in the frame of the old cell)
            float sum[3] = {0.0f, 0.0f, 0.0f};
            int lo[3] = {1 << 20, 1 << 20, 1 << 20}, hi[3] = {-(1 << 20), -(1 << 20), -(1 << 20)};
#pragma unroll 1
            for (int r = 0; r < kPerThread; ++r) {
                // consecutive particles: a warp's lanes sit in one to three cells,
                // so the gather reads the same or neighbouring window addresses
                const int q = 32 * (warp + kWarps * r) + lane;
                if (q >= cn) continue;
                const int sq = q + (q >> 5);
                if (BND && s_cell[sq] < 0) {   // left the box: kept as it is until the next sort
                    s_d[sq] = __int_as_float(0x7fc00000);
                    continue;
                }
                int cx, cy, cz;
                unpack_cell(s_cell[sq], cx, cy, cz);
                float xi0[3] = {s_o[sq], s_o[kStage + sq], s_o[2 * kStage + sq]};
                float u[3] = {s_u[sq], s_u[kStage + sq], s_u[2 * kStage + sq]};
                int rx = min_image(cx - ox, g.n[0]), ry = min_image(cy - oy, g.n[1]), rz = min_image(cz - oz, g.n[2]);
                bool inside = rx >= -kMargin && rx < kTile + kMargin && ry >= -kMargin && ry < kTile + kMargin &&
                              rz >= -kMargin && rz < kTile + kMargin;
                s_d[sq] = __int_as_float(0x7fc00000);   // not deposited here unless set below
                if (!inside) {   // drifted too far from the tile: leave it to the global-mesh kernel
                    unsigned slot = atomicAdd(S.slow_count, 1u);
                    S.slow_list[slot] = cb + q;
                    continue;
                }
                if (S.qmdt != 0.0f) {   // uniform: no kick, no force
                    float E[3], B[3];
                    SmemAcc sacc{F, Jw, win(rx + kWinLo, ry + kWinLo, rz + kWinLo)};
                    PP_IF_CHECKED(sacc.wx = rx + kWinLo; sacc.wy = ry + kWinLo; sacc.wz = rz + kWinLo; sacc.st = T.status;)
                    gather_EB<O, float>(sacc, xi0, E, B);
                    push_particle<PUSH, float>(S.qmdt, S.kdt, E, B, u);
                }
                float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                float dx[3];
                bool ok = true;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    dx[d] = T.dtdx[d] * u[d] * gi;
                    ok = ok && (fabsf(dx[d]) < 1.0f);
                }
                if (!ok) {   // leave the particle unchanged and flag the step
                    atomicOr(T.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
                    continue;
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    s_d[d * kStage + sq] = dx[d];
                    sum[d] += fabsf(dx[d]);
                }
                s_u[sq] = u[0]; s_u[kStage + sq] = u[1]; s_u[2 * kStage + sq] = u[2];
                lo[0] = min(lo[0], rx); lo[1] = min(lo[1], ry); lo[2] = min(lo[2], rz);
                hi[0] = max(hi[0], rx); hi[1] = max(hi[1], ry); hi[2] = max(hi[2], rz);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float sd = sum[d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
                int l = __reduce_min_sync(0xffffffffu, lo[d]), h = __reduce_max_sync(0xffffffffu, hi[d]);
                if (lane == 0) {
                    atomicAdd(tot + d, sd);
                    atomicMin(bbox + d, l);
                    atomicMax(bbox + 3 + d, h);
                }
            }
            __syncthreads();
            // ---- phase 2: fixed-point unit per component, deposit, re-bin
            float unit[3], jsc[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float bound = fixed_point_cy_bound<O>() * fabsf(S.jscale[d]) * (tot[d] + 1e-6f * (float)cn) * 1.001f;
                unit[d] = bound > 0.0f ? kFixedRange / bound : 0.0f;
                jsc[d] = S.jscale[d] * unit[d];
            }
            // The particle at staging index sq in the frame of its cell: old and
            // new offsets, and the accessor of its window position.
            auto frame = [&](int sq, float (&xi0)[3], float (&xi1)[3], int &cx, int &cy, int &cz) {
                unpack_cell(s_cell[sq], cx, cy, cz);
                for (int d = 0; d < 3; ++d) {
                    xi0[d] = s_o[d * kStage + sq];
                    xi1[d] = xi0[d] + s_d[d * kStage + sq];
                }
                int rx = min_image(cx - ox, g.n[0]), ry = min_image(cy - oy, g.n[1]), rz = min_image(cz - oz, g.n[2]);
                SmemAcc acc{F, Jw, win(rx + kWinLo, ry + kWinLo, rz + kWinLo)};
                PP_IF_CHECKED(acc.wx = rx + kWinLo; acc.wy = ry + kWinLo; acc.wz = rz + kWinLo; acc.st = T.status;)
                return acc;
            };
            auto finish = [&](int sq, float (&xi1)[3], int cx, int cy, int cz) {
                rebin(xi1[0], cx, g.n[0]);
                rebin(xi1[1], cy, g.n[1]);
                rebin(xi1[2], cz, g.n[2]);
                int32_t cw;
                if constexpr (BND) {
                    reflect(cx, xi1[0], s_u[sq], T.wall[0]);
                    reflect(cy, xi1[1], s_u[kStage + sq], T.wall[1]);
                    reflect(cz, xi1[2], s_u[2 * kStage + sq], T.wall[2]);
                    cw = pack_cell(cx, cy, cz);
                    if (T.esc > 0.0 && (double)cx + (double)xi1[0] < T.esc && s_u[sq] < 0.0f) cw |= kDeadBit;
                } else {
                    cw = pack_cell(cx, cy, cz);
                }
                s_cell[sq] = cw;
                s_o[sq] = xi1[0]; s_o[kStage + sq] = xi1[1]; s_o[2 * kStage + sq] = xi1[2];
            };
            // Most particles cross no support boundary in a step: they deposit
            // through the O (O+1)^2-site form.  The others are queued and then
            // deposited by all threads together, so that a warp's lanes take one
            // form at a time instead of every warp taking the union of both.
#pragma unroll 1
            for (int r = 0; r < kPerThread; ++r) {
                const int q = lane_q(lane, warp + kWarps * r, S.lane_shift);
                if (q >= cn) continue;
                const int sq = q + (q >> 5);
                if (isnan(s_d[sq])) continue;
                float xi0[3], xi1[3];
                int cx, cy, cz;
                SmemAcc sacc = frame(sq, xi0, xi1, cx, cy, cz);
                if (T.direct) {   // uniform: the direct current has one form for every particle
                    float dxs[3] = {s_d[sq], s_d[kStage + sq], s_d[2 * kStage + sq]};
                    deposit_direct<O, float>(sacc, xi0, dxs, jsc);
                    finish(sq, xi1, cx, cy, cz);
                    continue;
                }
                if (!deposit_esirkepov_inner<O, float>(sacc, xi0, xi1, jsc)) {
                    s_queue[atomicAdd(nqueue, 1)] = sq;
                    s_cell[sq] |= kQueued;   // re-binned when written back
                    continue;
                }
                finish(sq, xi1, cx, cy, cz);
            }
            __syncthreads();
            // The queue: groups of three warps take 32 particles per round, one
            // current component per warp (warps past the last group rest), so that the pass lasts
            // about a third of a deposit and no warp diverges over components.
            const int nq = *nqueue;
            const int group = warp / 3, comp = warp - 3 * group;
            if (group < kWarps / 3) {
#pragma unroll 1
                for (int k = 32 * group + lane; k < nq; k += 32 * (kWarps / 3)) {
                    const int sq = s_queue[k];
                    float xi0[3], xi1[3];
                    int cx, cy, cz;
                    SmemAcc sacc = frame(sq, xi0, xi1, cx, cy, cz);
                    float S0[3][O + 2], DS[3][O + 2];
                    int lo[3];
                    esirkepov_weights<O, float>(xi0, xi1, S0, DS, lo);
                    if (comp == 0) esirkepov_component<O, float, 0>(sacc, S0, DS, lo, jsc[0]);
                    else if (comp == 1) esirkepov_component<O, float, 1>(sacc, S0, DS, lo, jsc[1]);
                    else esirkepov_component<O, float, 2>(sacc, S0, DS, lo, jsc[2]);
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < cn; q += kThreads) {
                int sq = q + (q >> 5);
                if (s_cell[sq] & kQueued) {   // deposited from the queue: move it now
                    float xi0[3], xi1[3];
                    int cx, cy, cz;
                    frame(sq, xi0, xi1, cx, cy, cz);
                    finish(sq, xi1, cx, cy, cz);
                }
                S.p.cell[cb + q] = s_cell[sq];
                S.p.ox[cb + q] = s_o[sq]; S.p.oy[cb + q] = s_o[kStage + sq]; S.p.oz[cb + q] = s_o[2 * kStage + sq];
                S.p.ux[cb + q] = s_u[sq]; S.p.uy[cb + q] = s_u[kStage + sq]; S.p.uz[cb + q] = s_u[2 * kStage + sq];
            }
            // flush the window nodes this chunk could touch (cells +- support) into the FP32 mesh
            if (bbox[0] <= bbox[3]) {
                // box of window nodes, clamped to the window (deposited cells lie in
                // [-kMargin, kTile + kMargin) so the clamp never cuts real deposits)
                const int x0 = max(bbox[0] + kWinLo - kReachLo, 0), y0 = max(bbox[1] + kWinLo - kReachLo, 0),
                          z0 = max(bbox[2] + kWinLo - kReachLo, 0);
                const int ex = min(bbox[3] + kWinLo + kReachHi, kWin - 1) - x0 + 1;
                const int ey = min(bbox[4] + kWinLo + kReachHi, kWin - 1) - y0 + 1;
                const int ez = min(bbox[5] + kWinLo + kReachHi, kWin - 1) - z0 + 1;
                const int vol = ex * ey * ez;
                for (int idx = threadIdx.x; idx < 3 * vol; idx += kThreads) {
                    int comp = idx / vol, r = idx - comp * vol;
                    int i = x0 + r % ex, j = y0 + (r / ex) % ey, k = z0 + r / (ex * ey);
                    int w = win(i, j, k);
                    int iv = Jw[comp * kWinVol + w];
                    if (iv == 0) continue;
                    Jw[comp * kWinVol + w] = 0;
                    float uc = comp == 0 ? unit[0] : (comp == 1 ? unit[1] : unit[2]);
                    atomicAdd(T.J[comp] + g.at(wx + i, wy + j, wz + k), (float)iv / uc);
                }
            }
            __syncthreads();
        }
    }
}

// Particles the tile kernel left out (drifted more than kMargin cells from
// their tile since the last sort), advanced through the global mesh.
template <int O, int PUSH>
__global__ void __launch_bounds__(256) k_particles_listed(StepArgs<float> a, MixedParticles p, const int32_t *list,
                                                          const unsigned *count, unsigned long long *nslow) {
    unsigned n = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(nslow, (unsigned long long)n);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int t = list[k];
        if (p.cell[t] < 0) continue;
        int cx, cy, cz;
        unpack_cell(p.cell[t], cx, cy, cz);
        float xi0[3] = {p.ox[t], p.oy[t], p.oz[t]};
        float u[3] = {p.ux[t], p.uy[t], p.uz[t]};
        GlobalAcc<float> acc{a.g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, cx, cy, cz};
        PP_IF_CHECKED(acc.st = a.status;)
        if (a.qmdt != 0.0f) {
            float E[3], B[3];
            gather_EB<O, float>(acc, xi0, E, B);
            push_particle<PUSH, float>(a.qmdt, a.kdt, E, B, u);
        }
        float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        float xi1[3], dxs[3];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float dx = a.dtdx[d] * u[d] * gi;
            dxs[d] = dx;
            xi1[d] = xi0[d] + dx;
            ok = ok && (fabsf(dx) < 1.0f);
        }
        if (!ok) {
            atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
            continue;
        }
        if (a.direct) deposit_direct<O, float>(acc, xi0, dxs, a.jscale);
        else deposit_esirkepov<O, float>(acc, xi0, xi1, a.jscale);
        rebin(xi1[0], cx, a.g.n[0]);
        rebin(xi1[1], cy, a.g.n[1]);
        rebin(xi1[2], cz, a.g.n[2]);
        reflect(cx, xi1[0], u[0], a.wall[0]);
        reflect(cy, xi1[1], u[1], a.wall[1]);
        reflect(cz, xi1[2], u[2], a.wall[2]);
        int32_t cw = pack_cell(cx, cy, cz);
        if (a.esc > 0.0 && (double)cx + (double)xi1[0] < a.esc && u[0] < 0.0f) cw |= kDeadBit;
        p.cell[t] = cw;
        p.ox[t] = xi1[0]; p.oy[t] = xi1[1]; p.oz[t] = xi1[2];
        p.ux[t] = u[0]; p.uy[t] = u[1]; p.uz[t] = u[2];
    }
}

bool tiled_supported(const Ctx &c) {
    if (c.fp64 || c.g.G < kWinLo || c.g.G < kWin - kWinLo - kTile) return false;
    for (int a = 0; a < 3; ++a)
        if (c.g.n[a] % kTile != 0 || c.tile[a] != kTile) return false;
    return true;
}

// All species of the context in one launch (species with no particles skip
// their loop); fails if a species has not been sorted yet.
cudaError_t launch_particles_tiled_all(Ctx &c) {
    if (!tiled_supported(c)) return cudaErrorInvalidConfiguration;
    for (int s = 0; s < c.nspecies; ++s) {
        cudaError_t em = materialize(c, s);
        if (em != cudaSuccess) return em;
        c.sp[s].keys_valid = false;
    }
    TiledArgs T;
    T.g = c.g;
    double h[3] = {c.d.dx, c.d.dy, c.d.dz};
    for (int d = 0; d < 3; ++d) {
        T.E[d] = (const float *)c.E[d];
        T.B[d] = (const float *)c.B[d];
        T.J[d] = (float *)c.J[d];
        T.dtdx[d] = (float)(c.drift_dt / h[d]);
        T.nt[d] = c.ntile[d];
    }
    T.ns = 0;
    int sid[kMaxTiledSpecies];
    cudaError_t e0 = cudaMemsetAsync(c.d_slow_count, 0, sizeof(unsigned) * PP_MAX_SPECIES, c.st);
    if (e0 != cudaSuccess) return e0;
    for (int s = 0; s < c.nspecies; ++s) {
        const Species &S = c.sp[s];
        if (S.n == 0 || !S.sorted) continue;   // never sorted (only injected into): all of it is the tail
        sid[T.ns] = s;
        TiledSpecies &t = T.sp[T.ns++];
        t.p = MixedParticles{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        t.cell_start = S.cell_start;
        t.slow_list = S.keys;              // the sort keys are dead between sorts
        t.slow_count = c.d_slow_count + s;
        t.qmdt = (float)(S.q * c.kick_dt / S.m);
        t.kdt = (float)(c.kick_dt != 0.0 ? S.rad / c.kick_dt : 0.0);
        // lanes about one cell apart: the nearest power of two to the
        // species' mean particles per cell, 1..32
        double per_cell = (double)S.n / (double)c.g.cells();
        int sh = 0;
        while (sh < 5 && per_cell >= 1.5 * (double)(1 << sh)) ++sh;
        t.lane_shift = sh;
        for (int d = 0; d < 3; ++d) t.jscale[d] = (float)(-S.q * S.w * h[d] / c.drift_dt);
    }
    T.status = c.d_status;
    T.direct = c.current_mode == PP_CURRENT_DIRECT ? 1 : 0;
    for (int d = 0; d < 3; ++d) T.wall[d] = c.wall[d];
    T.esc = c.escape_now;
    unsigned blocks = (unsigned)(c.ntile[0] * c.ntile[1] * c.ntile[2]);
    int o = c.d.shape_order, pu = c.d.pusher;
    static unsigned long long attr_done[2][2][4] = {};
    const bool bnd = c.any_wall();
    cudaError_t e = cudaSuccess;
    if (T.ns > 0) {
#define PP_TB(O, PU, BD)                                                                                    \
    do {                                                                                                    \
        cudaError_t e_ = ensure_smem_attr(k_particles_tiled<O, PU, BD>, (int)kTiledSmem, attr_done[BD][PU][O]); \
        if (e_ != cudaSuccess) return e_;                                                                   \
        k_particles_tiled<O, PU, BD><<<blocks, kThreads, kTiledSmem, c.st>>>(T);                            \
    } while (0)
#define PP_T(O, PU)                                                                                         \
    do {                                                                                                    \
        if (bnd) PP_TB(O, PU, true); else PP_TB(O, PU, false);                                              \
    } while (0)
    if (pu == PP_BORIS) {
        if (o == 1) PP_T(1, PP_BORIS); else if (o == 2) PP_T(2, PP_BORIS); else PP_T(3, PP_BORIS);
    } else {
        if (o == 1) PP_T(1, PP_VAY); else if (o == 2) PP_T(2, PP_VAY); else PP_T(3, PP_VAY);
    }
#undef PP_T
#undef PP_TB
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the left-out particles of every species, on a fixed grid (count read on the device)
    for (int k = 0; k < T.ns; ++k) {
        const Species &S = c.sp[sid[k]];
        StepArgs<float> a = step_args<float>(c, sid[k]);
        MixedParticles p{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        const unsigned *cnt = c.d_slow_count + sid[k];
#define PP_S(O, PU) k_particles_listed<O, PU><<<304, 256, 0, c.st>>>(a, p, S.keys, cnt, c.d_nslow)
        if (pu == PP_BORIS) {
            if (o == 1) PP_S(1, PP_BORIS); else if (o == 2) PP_S(2, PP_BORIS); else PP_S(3, PP_BORIS);
        } else {
            if (o == 1) PP_S(1, PP_VAY); else if (o == 2) PP_S(2, PP_VAY); else PP_S(3, PP_VAY);
        }
#undef PP_S
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // particles injected since the sort (or into a never-sorted species): through the global mesh
    for (int s = 0; s < c.nspecies; ++s) {
        const Species &S = c.sp[s];
        const int64_t first = S.sorted ? S.nsorted : 0;
        if (S.n <= first) continue;
        StepArgs<float> a = step_args<float>(c, s);
        a.off = first;
        a.n = S.n - first;
        MixedParticles p{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        unsigned blocks = (unsigned)((a.n + 255) / 256);
#define PP_L(O, PU) k_particles_mixed<O, PU><<<blocks, 256, 0, c.st>>>(a, p)
        if (pu == PP_BORIS) {
            if (o == 1) PP_L(1, PP_BORIS); else if (o == 2) PP_L(2, PP_BORIS); else PP_L(3, PP_BORIS);
        } else {
            if (o == 1) PP_L(1, PP_VAY); else if (o == 2) PP_L(2, PP_VAY); else PP_L(3, PP_VAY);
        }
#undef PP_L
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Injection of inflow particles (Sec. V "Sliding window and injection of
// particles").  Draws come from the counter-based Philox4x32-10 generator of
// Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of the bijection
//   (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)),
// M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key advanced by 0x9E3779B9, 0xBB67AE85
// between rounds.  Particle i of a batch takes counter (i, 0, step, stream)
// under the 64-bit seed; each 32-bit word r gives the uniform (r + 1/2) 2^-32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * x[0], hi0 = __umulhi(0xD2511F53u, x[0]);
        const uint32_t lo1 = 0xCD9E8D57u * x[2], hi1 = __umulhi(0xCD9E8D57u, x[2]);
        const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
    }
}

__device__ __forceinline__ void uniforms4(uint64_t seed, uint32_t i, uint32_t step, uint32_t stream, double (&u)[4]) {
    uint32_t x[4] = {i, 0u, step, stream};
    philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
    for (int m = 0; m < 4; ++m) u[m] = ((double)x[m] + 0.5) * (1.0 / 4294967296.0);
}

struct InjectArgs {
    int64_t off, count;        // first slot, number of particles
    uint64_t seed;
    uint32_t step, pstream, vstream;
    double thick;              // slab thickness in x (physical)
    double ly, lz;             // box lengths in y and z
    double h[3];               // cell sizes
    int n[3];                  // mesh cells
    double u[3], u_th;         // drift proper velocity, thermal spread
    int mixed;
};

// Particle i: position (thick u0, Ly u1, Lz u2) from stream pstream, proper
// velocity drift + u_th (three Box-Muller normals) from stream vstream.
__global__ void k_inject(InjectArgs a, Fp64Particles p64, MixedParticles pm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    double U[4], V[4];
    uniforms4(a.seed, (uint32_t)i, a.step, a.pstream, U);
    uniforms4(a.seed, (uint32_t)i, a.step, a.vstream, V);
    const double X[3] = {a.thick * U[0], a.ly * U[1], a.lz * U[2]};
    const double r0 = sqrt(-2.0 * log(V[0])), r1 = sqrt(-2.0 * log(V[2]));
    const double g[3] = {r0 * cos(2.0 * M_PI * V[1]), r0 * sin(2.0 * M_PI * V[1]), r1 * cos(2.0 * M_PI * V[3])};
    const int64_t q = a.off + i;
    double xi[3];
    int cell[3];
    float o[3];
    for (int d = 0; d < 3; ++d) {
        double v = X[d] / a.h[d];
        if (v >= (double)a.n[d]) v -= (double)a.n[d];
        xi[d] = v;
        int ci = (int)floor(v);
        float of = (float)(v - ci);
        if (of >= 1.0f) { of = 0.0f; ci += 1; }
        if (ci >= a.n[d]) ci -= a.n[d];
        cell[d] = ci;
        o[d] = of;
    }
    const double u0 = a.u[0] + a.u_th * g[0], u1 = a.u[1] + a.u_th * g[1], u2 = a.u[2] + a.u_th * g[2];
    if (a.mixed) {
        pm.cell[q] = pack_cell(cell[0], cell[1], cell[2]);
        pm.ox[q] = o[0]; pm.oy[q] = o[1]; pm.oz[q] = o[2];
        pm.ux[q] = (float)u0; pm.uy[q] = (float)u1; pm.uz[q] = (float)u2;
    } else {
        p64.x[q] = xi[0]; p64.y[q] = xi[1]; p64.z[q] = xi[2];
        p64.ux[q] = u0; p64.uy[q] = u1; p64.uz[q] = u2;
    }
}

cudaError_t launch_inject(Ctx &c, int s, int64_t off, int64_t count, uint32_t step, uint32_t pstream, double thick) {
    if (count <= 0) return cudaSuccess;
    Species &S = c.sp[s];
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    S.keys_valid = false;
    const Ctx::Injector &I = c.inj[s];
    InjectArgs a;
    a.off = off;
    a.count = count;
    a.seed = I.seed;
    a.step = step;
    a.pstream = pstream;
    a.vstream = pstream + 1u + (uint32_t)s;
    a.thick = thick;
    a.ly = c.d.ny * c.d.dy;   // the physical box (the mesh is doubled on walled axes)
    a.lz = c.d.nz * c.d.dz;
    a.h[0] = c.d.dx; a.h[1] = c.d.dy; a.h[2] = c.d.dz;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = c.g.n[d];
        a.u[d] = I.u[d];
    }
    a.u_th = I.u_th;
    a.mixed = c.fp64 ? 0 : 1;
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_inject<<<(unsigned)((count + 255) / 256), 256, 0, c.st>>>(a, p64, pm);
    ++c.nlaunch;
    S.fresh = false;
    return cudaGetLastError();
}

// Sliding-window shift of the particles: every live particle moves one cell
// up in x; one that ends above the top wall (x > nw cells) leaves.
__global__ void k_window_particles(int64_t n, int nw, Fp64Particles p64, MixedParticles pm, int mixed) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (mixed) {
        int32_t cw = pm.cell[t];
        if (cw < 0) return;
        int cx, cy, cz;
        unpack_cell(cw, cx, cy, cz);
        ++cx;
        cw = pack_cell(cx, cy, cz);
        if (cx > nw || (cx == nw && pm.ox[t] > 0.0f)) cw |= kDeadBit;
        pm.cell[t] = cw;
    } else {
        double x = p64.x[t];
        if (x < 0.0) return;
        x += 1.0;
        p64.x[t] = x > (double)nw ? kDeadX : x;
    }
}

cudaError_t launch_window_particles(Ctx &c, int s) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    S.keys_valid = false;
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_window_particles<<<(unsigned)((S.n + 255) / 256), 256, 0, c.st>>>(S.n, c.wall[0], p64, pm, c.fp64 ? 0 : 1);
    ++c.nlaunch;
    S.fresh = false;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Charge density of eq:rho2 (FP64 accumulation on the compact mesh).
// ---------------------------------------------------------------------------
struct RhoAcc {
    Geom g;
    double *rho;
    int ox, oy, oz;
    __device__ __forceinline__ void addRho(int i, int j, int k, double v) const {
        int64_t q = wrap(ox + i, g.n[0]) + (int64_t)g.n[0] * (wrap(oy + j, g.n[1]) + (int64_t)g.n[1] * wrap(oz + k, g.n[2]));
        atomicAdd(rho + q, v);
    }
};

// Lane l of every warp takes particles from the l-th thirty-second of the
// (cell-sorted) array, so the lanes of a warp sit in distinct cells and their
// FP64 atomics do not pile onto the same nodes.
template <int O>
__global__ void k_rho(Geom g, double qw, int64_t n, int64_t off, Fp64Particles p64, MixedParticles pm, int mixed,
                      double *rho) {
    int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n32 = (n + 31) / 32;
    if (tt >= n32 * 32) return;
    int64_t t = (tt & 31) * n32 + (tt >> 5);
    if (t >= n) return;
    t += off;
    if (mixed ? pm.cell[t] < 0 : p64.x[t] < 0.0) return;   // left the box
    RhoAcc acc{g, rho, 0, 0, 0};
    double xi[3];
    if (mixed) {
        unpack_cell(pm.cell[t], acc.ox, acc.oy, acc.oz);
        xi[0] = pm.ox[t]; xi[1] = pm.oy[t]; xi[2] = pm.oz[t];
    } else {
        xi[0] = p64.x[t]; xi[1] = p64.y[t]; xi[2] = p64.z[t];
    }
    deposit_rho<O, double>(acc, xi, qw);
}

// Cell-sorted form: thread k owns cell k (its kSubKeys consecutive sort keys) and sums the eq:rho2
// weights of that cell's particles in FP64 registers over a fixed frame of
// nodes around the cell, then adds the frame to the mesh once, instead of
// once per particle.  A particle that moved to another cell since the sort
// is added directly.
struct RhoCellGeom {
    int T[3];
    int nt[3];
    int tile_vol;
};

// A (accumulation type) is double for FP64 contexts and float for the mixed
// form, whose positions are FP32 already; the mesh sum stays FP64.
template <int O, typename A>
__global__ void __launch_bounds__(128) k_rho_cells(Geom g, RhoCellGeom kg, int64_t nkeys, const int32_t *cell_start,
                                                   double qw, Fp64Particles p64, MixedParticles pm, int mixed,
                                                   double *rho) {
    constexpr bool odd = (O % 2) == 1;
    constexpr int NF = odd ? O + 1 : O + 2;         // frame nodes per axis
    constexpr int ST = odd ? -(O - 1) / 2 : -O / 2; // frame start relative to the cell
    int64_t key = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= nkeys) return;
    const int b = cell_start[key * kSubKeys], e = cell_start[(key + 1) * kSubKeys];
    if (b == e) return;
    int tile = (int)(key / kg.tile_vol), loc = (int)(key % kg.tile_vol);
    int c0 = (tile % kg.nt[0]) * kg.T[0] + loc % kg.T[0];
    int c1 = ((tile / kg.nt[0]) % kg.nt[1]) * kg.T[1] + (loc / kg.T[0]) % kg.T[1];
    int c2 = (tile / (kg.nt[0] * kg.nt[1])) * kg.T[2] + loc / (kg.T[0] * kg.T[1]);
    A acc[NF][NF][NF];
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NF; ++j)
#pragma unroll
            for (int i = 0; i < NF; ++i) acc[k][j][i] = A(0);
    for (int t = b; t < e; ++t) {
        int cx, cy, cz;
        double xi[3];
        if (mixed ? pm.cell[t] < 0 : p64.x[t] < 0.0) continue;   // left the box
        if (mixed) {
            unpack_cell(pm.cell[t], cx, cy, cz);
            xi[0] = pm.ox[t]; xi[1] = pm.oy[t]; xi[2] = pm.oz[t];
        } else {
            double X[3] = {p64.x[t], p64.y[t], p64.z[t]};
            int cc[3];
            for (int a = 0; a < 3; ++a) {
                cc[a] = min(max((int)floor(X[a]), 0), g.n[a] - 1);
                xi[a] = X[a] - cc[a];
            }
            cx = cc[0]; cy = cc[1]; cz = cc[2];
        }
        if (cx != c0 || cy != c1 || cz != c2) {   // left its sorted cell: add it directly
            RhoAcc acc1{g, rho, cx, cy, cz};
            deposit_rho<O, double>(acc1, xi, qw);
            continue;
        }
        A w[3][NF];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A ws[O + 1];
            int sh = support<O, A>((A)xi[a], false, ws) - ST;   // 0, or 1 for even orders
#pragma unroll
            for (int m = 0; m < NF; ++m) w[a][m] = (m - sh >= 0 && m - sh <= O) ? ws[m - sh] : A(0);
        }
#pragma unroll
        for (int k = 0; k < NF; ++k)
#pragma unroll
            for (int j = 0; j < NF; ++j) {
                A wjk = w[1][j] * w[2][k];
#pragma unroll
                for (int i = 0; i < NF; ++i) acc[k][j][i] += w[0][i] * wjk;
            }
    }
    RhoAcc out{g, rho, c0, c1, c2};
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NF; ++j)
#pragma unroll
            for (int i = 0; i < NF; ++i)
                if (acc[k][j][i] != A(0)) out.addRho(ST + i, ST + j, ST + k, qw * (double)acc[k][j][i]);
}

// Mixed form, one CTA per sort tile, one thread per cell: each thread sums its
// cell's particles into an FP32 frame of NF^3 nodes in registers (as
// k_rho_cells), the frames go to shared memory, and each node of the tile's
// window (the tile plus the frames' reach) adds up the frames that cover it,
// in FP64, before one global atomic.  Global atomics per tile: the window's
// nodes instead of NF^3 per cell.
// A particle that left its sorted cell, deposited on its own (kept out of line
// so that its registers do not add to the frame loop's).
template <int O>
__device__ __noinline__ void rho_direct(Geom g, double *rho, int cx, int cy, int cz, double x0, double x1, double x2,
                                        double qw) {
    RhoAcc acc1{g, rho, cx, cy, cz};
    double xi[3] = {x0, x1, x2};
    deposit_rho<O, double>(acc1, xi, qw);
}

template <int O>
__global__ void __launch_bounds__(512) k_rho_tile(Geom g, RhoCellGeom kg, const int32_t *cell_start, double qw,
                                                  MixedParticles pm, double *rho) {
    constexpr bool odd = (O % 2) == 1;
    constexpr int NF = odd ? O + 1 : O + 2;         // frame nodes per axis
    constexpr int ST = odd ? -(O - 1) / 2 : -O / 2; // frame start relative to the cell
    constexpr int F3 = NF * NF * NF, FP = F3 + 1;   // frame size; padded pitch (distinct banks per cell)
    extern __shared__ float fr[];
    const int tile = blockIdx.x, loc = threadIdx.x;
    const int T0 = kg.T[0], T1 = kg.T[1], T2 = kg.T[2];
    const int lx = loc % T0, ly = (loc / T0) % T1, lz = loc / (T0 * T1);
    const int ox = (tile % kg.nt[0]) * T0, oy = ((tile / kg.nt[0]) % kg.nt[1]) * T1,
              oz = (tile / (kg.nt[0] * kg.nt[1])) * T2;
    const int c0 = ox + lx, c1 = oy + ly, c2 = oz + lz;
    const int64_t key = (int64_t)tile * kg.tile_vol + loc;
    const int b = cell_start[key * kSubKeys], e = cell_start[(key + 1) * kSubKeys];
    float acc[NF][NF][NF];
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NF; ++j)
#pragma unroll
            for (int i = 0; i < NF; ++i) acc[k][j][i] = 0.0f;
    for (int t = b; t < e; ++t) {
        const int32_t cw = pm.cell[t];
        if (cw < 0) continue;   // left the box
        int cx, cy, cz;
        unpack_cell(cw, cx, cy, cz);
        if (cx != c0 || cy != c1 || cz != c2) continue;   // left its sorted cell: second pass
        const float xi[3] = {pm.ox[t], pm.oy[t], pm.oz[t]};
        float w[3][NF];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float ws[O + 1];
            const int sh = support<O, float>(xi[a], false, ws) - ST;   // 0, or 1 for even orders
#pragma unroll
            for (int m = 0; m < NF; ++m) w[a][m] = (m - sh >= 0 && m - sh <= O) ? ws[m - sh] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < NF; ++k)
#pragma unroll
            for (int j = 0; j < NF; ++j) {
                const float wjk = w[1][j] * w[2][k];
#pragma unroll
                for (int i = 0; i < NF; ++i) acc[k][j][i] += w[0][i] * wjk;
            }
    }
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NF; ++j)
#pragma unroll
            for (int i = 0; i < NF; ++i) fr[loc * FP + (k * NF + j) * NF + i] = acc[k][j][i];
    for (int t = b; t < e; ++t) {   // particles that left their sorted cell, added directly
        const int32_t cw = pm.cell[t];
        if (cw < 0) continue;
        int cx, cy, cz;
        unpack_cell(cw, cx, cy, cz);
        if (cx != c0 || cy != c1 || cz != c2) rho_direct<O>(g, rho, cx, cy, cz, pm.ox[t], pm.oy[t], pm.oz[t], qw);
    }
    __syncthreads();
    // window node (wx, wy, wz) is mesh node (ox + ST + wx, ...); cell l of the
    // tile reaches it with frame index w - l
    const int W0 = T0 + NF - 1, W1 = T1 + NF - 1, W2 = T2 + NF - 1;
    for (int nd = threadIdx.x; nd < W0 * W1 * W2; nd += blockDim.x) {
        const int wx = nd % W0, wy = (nd / W0) % W1, wz = nd / (W0 * W1);
        double sum = 0.0;
        for (int k = max(0, wz - T2 + 1); k <= min(NF - 1, wz); ++k)
            for (int j = max(0, wy - T1 + 1); j <= min(NF - 1, wy); ++j)
                for (int i = max(0, wx - T0 + 1); i <= min(NF - 1, wx); ++i) {
                    const int cell = ((wz - k) * T1 + (wy - j)) * T0 + (wx - i);
                    sum += (double)fr[cell * FP + (k * NF + j) * NF + i];
                }
        if (sum != 0.0) {
            RhoAcc out{g, rho, ox + ST, oy + ST, oz + ST};
            out.addRho(wx, wy, wz, qw * sum);
        }
    }
}

cudaError_t launch_rho(Ctx &c, bool sort_first) {
    for (int s = 0; s < c.nspecies; ++s) {
        const Species &S = c.sp[s];
        if (sort_first && !c.fp64 && S.n > 0 && (S.keys_valid || !S.sorted)) {
            cudaError_t es = launch_sort(c, s);
            if (es != cudaSuccess) return es;
        }
        cudaError_t em = materialize(c, s);
        if (em != cudaSuccess) return em;
    }
    cudaError_t e = cudaMemsetAsync(c.rho, 0, sizeof(double) * c.g.cells(), c.st);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < c.nspecies; ++s) {
        Species &S = c.sp[s];
        if (S.n == 0) continue;
        Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
        MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        double qw = S.q * S.w;
        int mixed = c.fp64 ? 0 : 1;
        if (S.sorted) {
            RhoCellGeom kg;
            for (int a = 0; a < 3; ++a) {
                kg.T[a] = c.tile[a];
                kg.nt[a] = c.ntile[a];
            }
            kg.tile_vol = c.tile[0] * c.tile[1] * c.tile[2];
            int64_t ncell = c.nkeys / kSubKeys;
            unsigned kb = (unsigned)((ncell + 127) / 128);
#define PP_R(O, A) k_rho_cells<O, A><<<kb, 128, 0, c.st>>>(c.g, kg, ncell, S.cell_start, qw, p64, pm, mixed, c.rho)
#define PP_T(O)                                                                                            \
    do {                                                                                                   \
        constexpr int nf = (O % 2) ? O + 1 : O + 2;                                                       \
        const size_t sm = sizeof(float) * (size_t)kg.tile_vol * (nf * nf * nf + 1);                        \
        static unsigned long long attr = 0;                                                               \
        cudaError_t e_ = ensure_smem_attr(k_rho_tile<O>, (int)(sizeof(float) * 512 * (nf * nf * nf + 1)), attr); \
        if (e_ != cudaSuccess) return e_;                                                                  \
        k_rho_tile<O><<<(unsigned)(c.ntile[0] * c.ntile[1] * c.ntile[2]), kg.tile_vol, sm, c.st>>>(       \
            c.g, kg, S.cell_start, qw, pm, c.rho);                                                         \
    } while (0)
            if (mixed) {
                if (c.d.shape_order == 1) PP_T(1); else if (c.d.shape_order == 2) PP_T(2); else PP_T(3);
            } else {
                if (c.d.shape_order == 1) PP_R(1, double); else if (c.d.shape_order == 2) PP_R(2, double); else PP_R(3, double);
            }
#undef PP_R
#undef PP_T
            ++c.nlaunch;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // every particle of an unsorted species, or the unsorted tail (injected since the sort)
        const int64_t off = S.sorted ? S.nsorted : 0, cnt = S.n - off;
        if (cnt <= 0) continue;
        unsigned blocks = (unsigned)(((cnt + 31) / 32 * 32 + 255) / 256);
        if (c.d.shape_order == 1) k_rho<1><<<blocks, 256, 0, c.st>>>(c.g, qw, cnt, off, p64, pm, mixed, c.rho);
        else if (c.d.shape_order == 2) k_rho<2><<<blocks, 256, 0, c.st>>>(c.g, qw, cnt, off, p64, pm, mixed, c.rho);
        else k_rho<3><<<blocks, 256, 0, c.st>>>(c.g, qw, cnt, off, p64, pm, mixed, c.rho);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return launch_mirror_rho(c, c.rho);   // between walls: add the virtual images' charge
}

// ---------------------------------------------------------------------------
// Kinetic energy sum_p w m (gamma - 1) dV (FP64).
// ---------------------------------------------------------------------------
__global__ void k_kinetic(int64_t n, Fp64Particles p64, MixedParticles pm, int mixed, double scale, double *out) {
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double u0, u1, u2;
        if (mixed ? pm.cell[t] < 0 : p64.x[t] < 0.0) continue;   // left the box
        if (mixed) { u0 = pm.ux[t]; u1 = pm.uy[t]; u2 = pm.uz[t]; }
        else { u0 = p64.ux[t]; u1 = p64.uy[t]; u2 = p64.uz[t]; }
        double u2s = u0 * u0 + u1 * u1 + u2 * u2;
        acc += u2s / (sqrt(1.0 + u2s) + 1.0);   // gamma - 1 without cancellation
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(out, acc * scale);
    }
}

cudaError_t launch_kinetic(Ctx &c, double *out) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * PP_MAX_SPECIES, c.st);
    if (e != cudaSuccess) return e;
    double dV = c.d.dx * c.d.dy * c.d.dz;
    for (int s = 0; s < c.nspecies; ++s) {
        Species &S = c.sp[s];
        if (S.n == 0) continue;
        Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
        MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        int64_t want = (S.n + 255) / 256;
        unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
        k_kinetic<<<blocks, 256, 0, c.st>>>(S.n, p64, pm, c.fp64 ? 0 : 1, S.w * S.m * dV, out + s);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Conversions between the ABI's FP64 physical arrays and the storage forms.
// ---------------------------------------------------------------------------
// Reads each input once (from device memory, or from pinned host memory over
// the host link) and flags a non-finite value in *bad instead of storing it.
__global__ void k_convert_in(int64_t n, int64_t off, const double *x, const double *y, const double *z,
                             const double *ux, const double *uy, const double *uz, double hx, double hy,
                             double hz, int nx, int ny, int nz, int mixed, Fp64Particles p64, MixedParticles pm,
                             int *bad, double wx, double wy, double wz) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double in[3] = {x[t], y[t], z[t]};
    const double vx = ux[t], vy = uy[t], vz = uz[t];
    if (!isfinite(in[0]) || !isfinite(in[1]) || !isfinite(in[2]) || !isfinite(vx) || !isfinite(vy) || !isfinite(vz)) {
        atomicOr(bad, 1);
        return;
    }
    const double wl[3] = {wx, wy, wz};   // walls at 0 and L_a on axes with L_a > 0
    for (int d = 0; d < 3; ++d)
        if (wl[d] > 0.0 && !(in[d] >= 0.0 && in[d] <= wl[d])) {
            atomicOr(bad, 2);
            return;
        }
    double h[3] = {hx, hy, hz};
    int N[3] = {nx, ny, nz};
    double xi[3];
    int cell[3];
    float o[3];
    for (int d = 0; d < 3; ++d) {
        double v = in[d] / h[d];
        v -= (double)N[d] * floor(v / (double)N[d]);
        if (v >= (double)N[d]) v -= (double)N[d];
        if (v < 0.0) v = 0.0;
        xi[d] = v;
        int ci = (int)floor(v);
        float of = (float)(v - ci);
        if (of >= 1.0f) { of = 0.0f; ci += 1; }
        if (ci >= N[d]) ci -= N[d];
        cell[d] = ci;
        o[d] = of;
    }
    int64_t q = off + t;
    if (mixed) {
        pm.cell[q] = pack_cell(cell[0], cell[1], cell[2]);
        pm.ox[q] = o[0]; pm.oy[q] = o[1]; pm.oz[q] = o[2];
        pm.ux[q] = (float)vx; pm.uy[q] = (float)vy; pm.uz[q] = (float)vz;
    } else {
        p64.x[q] = xi[0]; p64.y[q] = xi[1]; p64.z[q] = xi[2];
        p64.ux[q] = vx; p64.uy[q] = vy; p64.uz[q] = vz;
    }
}

cudaError_t launch_convert_in(Ctx &c, int s, int64_t off, int64_t n, const double *x, const double *y,
                              const double *z, const double *ux, const double *uy, const double *uz, int *bad) {
    if (n == 0) return cudaSuccess;
    Species &S = c.sp[s];
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    S.keys_valid = false;
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_convert_in<<<(unsigned)((n + 255) / 256), 256, 0, c.st>>>(n, off, x, y, z, ux, uy, uz, c.d.dx, c.d.dy, c.d.dz,
                                                               c.g.n[0], c.g.n[1], c.g.n[2], c.fp64 ? 0 : 1, p64, pm,
                                                               bad, c.wall[0] * c.d.dx, c.wall[1] * c.d.dy,
                                                               c.wall[2] * c.d.dz);
    ++c.nlaunch;
    return cudaGetLastError();
}

__global__ void k_convert_out(int64_t n, double hx, double hy, double hz, int mixed, Fp64Particles p64,
                              MixedParticles pm, double *x, double *y, double *z, double *ux, double *uy, double *uz) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (mixed) {
        int cx, cy, cz;
        unpack_cell(pm.cell[t], cx, cy, cz);
        x[t] = ((double)cx + (double)pm.ox[t]) * hx;
        y[t] = ((double)cy + (double)pm.oy[t]) * hy;
        z[t] = ((double)cz + (double)pm.oz[t]) * hz;
        ux[t] = pm.ux[t]; uy[t] = pm.uy[t]; uz[t] = pm.uz[t];
    } else {
        x[t] = p64.x[t] * hx; y[t] = p64.y[t] * hy; z[t] = p64.z[t] * hz;
        ux[t] = p64.ux[t]; uy[t] = p64.uy[t]; uz[t] = p64.uz[t];
    }
}

cudaError_t launch_convert_out(Ctx &c, int s, double *x, double *y, double *z, double *ux, double *uy, double *uz) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_convert_out<<<(unsigned)((S.n + 255) / 256), 256, 0, c.st>>>(S.n, c.d.dx, c.d.dy, c.d.dz, c.fp64 ? 0 : 1,
                                                                   p64, pm, x, y, z, ux, uy, uz);
    ++c.nlaunch;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Particles of a z-slab decomposition that moved out of the slab
// [z_lo, z_hi) (physical z): counted (write = 0), or written out as FP64
// physical state and marked as gone (write = 1, the first `cap` of them).
// ---------------------------------------------------------------------------
__global__ void k_extract(int64_t n, double hx, double hy, double hz, double z_lo, double z_hi, int mixed, int write,
                          int64_t cap, Fp64Particles p64, MixedParticles pm, unsigned long long *count, double *x,
                          double *y, double *z, double *ux, double *uy, double *uz) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double px, py, pz;
    if (mixed) {
        const int32_t cw = pm.cell[t];
        if (cw < 0) return;   // gone already
        int cx, cy, cz;
        unpack_cell(cw, cx, cy, cz);
        px = ((double)cx + (double)pm.ox[t]) * hx;
        py = ((double)cy + (double)pm.oy[t]) * hy;
        pz = ((double)cz + (double)pm.oz[t]) * hz;
    } else {
        if (p64.x[t] < 0.0) return;
        px = p64.x[t] * hx; py = p64.y[t] * hy; pz = p64.z[t] * hz;
    }
    if (pz >= z_lo && pz < z_hi) return;
    const unsigned long long slot = atomicAdd(count, 1ull);
    if (!write || slot >= (unsigned long long)cap) return;
    x[slot] = px; y[slot] = py; z[slot] = pz;
    if (mixed) {
        ux[slot] = pm.ux[t]; uy[slot] = pm.uy[t]; uz[slot] = pm.uz[t];
        pm.cell[t] |= kDeadBit;
    } else {
        ux[slot] = p64.ux[t]; uy[slot] = p64.uy[t]; uz[slot] = p64.uz[t];
        p64.x[t] = kDeadX;
    }
}

cudaError_t launch_extract(Ctx &c, int s, double z_lo, double z_hi, int write, int64_t cap,
                           unsigned long long *count, double *const out[6]) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    cudaError_t em = materialize(c, s);
    if (em != cudaSuccess) return em;
    if (write) S.keys_valid = false;
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_extract<<<(unsigned)((S.n + 255) / 256), 256, 0, c.st>>>(S.n, c.d.dx, c.d.dy, c.d.dz, z_lo, z_hi,
                                                               c.fp64 ? 0 : 1, write, cap, p64, pm, count, out[0],
                                                               out[1], out[2], out[3], out[4], out[5]);
    ++c.nlaunch;
    return cudaGetLastError();
}

}  // namespace pp
