// pp_particles.cu -- per-particle kernels: the fused gather -> push -> move ->
// charge-conserving deposit (Sec. III steps 1-3) in its one-thread-per-particle
// form, the charge density of eq:rho2, the kinetic-energy reduction and the
// FP64 <-> storage conversions of pp_load_particles / pp_get_particles.
#include "pp_internal.cuh"

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
    __device__ __forceinline__ R F(int kind, int comp, int i, int j, int k) const {
        const R *p = kind ? B[comp] : E[comp];
        return __ldg(p + g.at(ox + i, oy + j, oz + k));
    }
    __device__ __forceinline__ void addJ(int comp, int i, int j, int k, R v) const {
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
    R dtdx[3];
    R jscale[3];
    int64_t n;
    int *status;
};

struct Fp64Particles {
    double *x, *y, *z, *ux, *uy, *uz;
};

struct MixedParticles {
    int32_t *cell;
    float *ox, *oy, *oz, *ux, *uy, *uz;
};

template <int O, int PUSH>
__global__ void __launch_bounds__(256) k_particles_fp64(StepArgs<double> a, Fp64Particles p) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    double xi0[3] = {p.x[t], p.y[t], p.z[t]};
    double u[3] = {p.ux[t], p.uy[t], p.uz[t]};
    GlobalAcc<double> acc{a.g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, 0, 0, 0};
    double E[3], B[3];
    gather_EB<O, double>(acc, xi0, E, B);
    if (PUSH == PP_BORIS) push_boris<double>(a.qmdt, E, B, u);
    else push_vay<double>(a.qmdt, E, B, u);
    double gi = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double xi1[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double dx = a.dtdx[d] * u[d] * gi;
        xi1[d] = xi0[d] + dx;
        ok = ok && (fabs(dx) < 1.0);   // also false for NaN
    }
    if (!ok) {
        atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
        return;
    }
    deposit_esirkepov<O, double>(acc, xi0, xi1, a.jscale);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double L = (double)a.g.n[d], v = xi1[d];
        if (v < 0.0) v += L;
        else if (v >= L) v -= L;
        if (v >= L) v -= L;
        xi1[d] = v;
    }
    p.x[t] = xi1[0]; p.y[t] = xi1[1]; p.z[t] = xi1[2];
    p.ux[t] = u[0]; p.uy[t] = u[1]; p.uz[t] = u[2];
}

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

template <int O, int PUSH>
__global__ void __launch_bounds__(256) k_particles_mixed(StepArgs<float> a, MixedParticles p) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    int cx, cy, cz;
    unpack_cell(p.cell[t], cx, cy, cz);
    float xi0[3] = {p.ox[t], p.oy[t], p.oz[t]};
    float u[3] = {p.ux[t], p.uy[t], p.uz[t]};
    GlobalAcc<float> acc{a.g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, cx, cy, cz};
    float E[3], B[3];
    gather_EB<O, float>(acc, xi0, E, B);
    if (PUSH == PP_BORIS) push_boris<float>(a.qmdt, E, B, u);
    else push_vay<float>(a.qmdt, E, B, u);
    float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    float xi1[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float dx = a.dtdx[d] * u[d] * gi;
        xi1[d] = xi0[d] + dx;
        ok = ok && (fabsf(dx) < 1.0f);
    }
    if (!ok) {
        atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
        return;
    }
    deposit_esirkepov<O, float>(acc, xi0, xi1, a.jscale);
    rebin(xi1[0], cx, a.g.n[0]);
    rebin(xi1[1], cy, a.g.n[1]);
    rebin(xi1[2], cz, a.g.n[2]);
    p.cell[t] = pack_cell(cx, cy, cz);
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
    a.qmdt = (R)(S.q * c.d.dt / S.m);
    for (int d = 0; d < 3; ++d) {
        a.dtdx[d] = (R)(c.d.dt / h[d]);
        a.jscale[d] = (R)(-S.q * S.w * h[d] / c.d.dt);
    }
    a.n = S.n;
    a.status = c.d_status;
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
// sort; the E/B nodes the tile's particles can touch are staged in shared
// memory, the current is accumulated in a shared tile and flushed to the
// global mesh once.  Thread t owns cell t of the tile and walks that cell's
// sorted particle range, so the 32 lanes of a warp sit in 32 distinct cells
// and their shared-memory atomics hit distinct addresses.
//
// A particle may have drifted since the sort: it is handled from shared
// memory while its cell lies within kMargin cells of the tile (minimal
// periodic image), otherwise through the global mesh (counted in n_slow).
// ---------------------------------------------------------------------------
constexpr int kTile = 8;                       // tile edge (cells)
constexpr int kMargin = 2;                     // drift allowed before the fallback
constexpr int kReachLo = 2, kReachHi = 3;      // deposit/gather reach around a cell
constexpr int kWin = kTile + 2 * kMargin + kReachLo + kReachHi;   // 17 nodes per axis
constexpr int kWin3 = kWin * kWin * kWin;
constexpr int kWinLo = kMargin + kReachLo;     // window node 0 = tile origin - kWinLo
constexpr size_t kTiledSmem = sizeof(float) * 9 * kWin3;

struct SmemAcc {
    const float *Fw;  // 6 windows: E0 E1 E2 B0 B1 B2
    float *J;         // 3 windows
    int fx, fy, fz;   // window index of the particle's cell
    __device__ __forceinline__ int at(int i, int j, int k) const {
        return ((k + fz) * kWin + (j + fy)) * kWin + (i + fx);
    }
    __device__ __forceinline__ float F(int kind, int comp, int i, int j, int k) const {
        return Fw[(kind * 3 + comp) * kWin3 + at(i, j, k)];
    }
    __device__ __forceinline__ void addJ(int comp, int i, int j, int k, float v) const {
        atomicAdd(J + comp * kWin3 + at(i, j, k), v);
    }
};

struct TiledArgs {
    StepArgs<float> a;
    MixedParticles p;
    const int32_t *cell_start;   // per sort key, tile-major
    int nt[3];                   // tiles per axis
    unsigned long long *nslow;
};

__device__ __forceinline__ int min_image(int d, int n) {
    if (d > n / 2) d -= n;
    else if (d < -(n / 2)) d += n;
    return d;
}

template <int O, int PUSH>
__global__ void __launch_bounds__(kTile * kTile * kTile, 1) k_particles_tiled(TiledArgs T) {
    extern __shared__ float smem[];
    float *F = smem;
    float *Jw = smem + 6 * kWin3;
    const StepArgs<float> &a = T.a;
    const Geom &g = a.g;
    int tile = blockIdx.x;
    int tx = tile % T.nt[0], ty = (tile / T.nt[0]) % T.nt[1], tz = tile / (T.nt[0] * T.nt[1]);
    int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
    int wx = ox - kWinLo, wy = oy - kWinLo, wz = oz - kWinLo;
    // stage E and B (ghost layers hold the periodic images), clear the current window
    for (int idx = threadIdx.x; idx < 6 * kWin3; idx += blockDim.x) {
        int comp = idx / kWin3, r = idx - comp * kWin3;
        int i = r % kWin, j = (r / kWin) % kWin, k = r / (kWin * kWin);
        const float *src = comp < 3 ? a.E[comp] : a.B[comp - 3];
        F[idx] = __ldg(src + g.at(wx + i, wy + j, wz + k));
    }
    for (int idx = threadIdx.x; idx < 3 * kWin3; idx += blockDim.x) Jw[idx] = 0.0f;
    __syncthreads();

    int lc = threadIdx.x;
    int key = tile * (kTile * kTile * kTile) + lc;
    int begin = T.cell_start[key], end = T.cell_start[key + 1];
    GlobalAcc<float> gacc{g, {a.E[0], a.E[1], a.E[2]}, {a.B[0], a.B[1], a.B[2]}, {a.J[0], a.J[1], a.J[2]}, 0, 0, 0};
    for (int t = begin; t < end; ++t) {
        int cx, cy, cz;
        unpack_cell(T.p.cell[t], cx, cy, cz);
        float xi0[3] = {T.p.ox[t], T.p.oy[t], T.p.oz[t]};
        float u[3] = {T.p.ux[t], T.p.uy[t], T.p.uz[t]};
        int rx = min_image(cx - ox, g.n[0]), ry = min_image(cy - oy, g.n[1]), rz = min_image(cz - oz, g.n[2]);
        bool inside = rx >= -kMargin && rx < kTile + kMargin && ry >= -kMargin && ry < kTile + kMargin &&
                      rz >= -kMargin && rz < kTile + kMargin;
        float E[3], B[3];
        SmemAcc sacc{F, Jw, rx + kWinLo, ry + kWinLo, rz + kWinLo};
        gacc.ox = cx; gacc.oy = cy; gacc.oz = cz;
        if (inside) gather_EB<O, float>(sacc, xi0, E, B);
        else gather_EB<O, float>(gacc, xi0, E, B);
        if (PUSH == PP_BORIS) push_boris<float>(a.qmdt, E, B, u);
        else push_vay<float>(a.qmdt, E, B, u);
        float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        float xi1[3];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float dx = a.dtdx[d] * u[d] * gi;
            xi1[d] = xi0[d] + dx;
            ok = ok && (fabsf(dx) < 1.0f);
        }
        if (!ok) {
            atomicOr(a.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
            continue;
        }
        if (inside) {
            deposit_esirkepov<O, float>(sacc, xi0, xi1, a.jscale);
        } else {
            deposit_esirkepov<O, float>(gacc, xi0, xi1, a.jscale);
            atomicAdd(T.nslow, 1ull);
        }
        rebin(xi1[0], cx, g.n[0]);
        rebin(xi1[1], cy, g.n[1]);
        rebin(xi1[2], cz, g.n[2]);
        T.p.cell[t] = pack_cell(cx, cy, cz);
        T.p.ox[t] = xi1[0]; T.p.oy[t] = xi1[1]; T.p.oz[t] = xi1[2];
        T.p.ux[t] = u[0]; T.p.uy[t] = u[1]; T.p.uz[t] = u[2];
    }
    __syncthreads();
    // one flush of the current window into the global mesh (ghosts folded later)
    for (int idx = threadIdx.x; idx < 3 * kWin3; idx += blockDim.x) {
        float v = Jw[idx];
        if (v == 0.0f) continue;
        int comp = idx / kWin3, r = idx - comp * kWin3;
        int i = r % kWin, j = (r / kWin) % kWin, k = r / (kWin * kWin);
        atomicAdd(a.J[comp] + g.at(wx + i, wy + j, wz + k), v);
    }
}

bool tiled_supported(const Ctx &c) {
    for (int a = 0; a < 3; ++a)
        if (c.g.n[a] % kTile != 0 || c.tile[a] != kTile || c.g.G < kWinLo || c.g.G + 1 < kWin - kWinLo - kTile + 1)
            return false;
    return !c.fp64;
}

cudaError_t launch_particles_mixed_tiled(Ctx &c, int s) {
    Species &S = c.sp[s];
    if (S.n == 0) return cudaSuccess;
    if (!tiled_supported(c) || !S.sorted) return cudaErrorInvalidConfiguration;
    TiledArgs T;
    T.a = step_args<float>(c, s);
    T.p = MixedParticles{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    T.cell_start = S.cell_start;
    for (int a = 0; a < 3; ++a) T.nt[a] = c.ntile[a];
    T.nslow = c.d_nslow;
    unsigned blocks = (unsigned)(c.ntile[0] * c.ntile[1] * c.ntile[2]);
    int o = c.d.shape_order, pu = c.d.pusher;
    static bool attr_done[2][4] = {{false}};
#define PP_T(O, PU)                                                                                         \
    do {                                                                                                    \
        if (!attr_done[PU][O]) {                                                                            \
            cudaError_t e_ = cudaFuncSetAttribute(k_particles_tiled<O, PU>,                                 \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTiledSmem); \
            if (e_ != cudaSuccess) return e_;                                                               \
            attr_done[PU][O] = true;                                                                        \
        }                                                                                                   \
        k_particles_tiled<O, PU><<<blocks, kTile * kTile * kTile, kTiledSmem, c.st>>>(T);                   \
    } while (0)
    if (pu == PP_BORIS) {
        if (o == 1) PP_T(1, PP_BORIS); else if (o == 2) PP_T(2, PP_BORIS); else PP_T(3, PP_BORIS);
    } else {
        if (o == 1) PP_T(1, PP_VAY); else if (o == 2) PP_T(2, PP_VAY); else PP_T(3, PP_VAY);
    }
#undef PP_T
    ++c.nlaunch;
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

template <int O>
__global__ void k_rho(Geom g, double qw, int64_t n, Fp64Particles p64, MixedParticles pm, int mixed, double *rho) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
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

cudaError_t launch_rho(Ctx &c) {
    cudaError_t e = cudaMemsetAsync(c.rho, 0, sizeof(double) * c.g.cells(), c.st);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < c.nspecies; ++s) {
        Species &S = c.sp[s];
        if (S.n == 0) continue;
        Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
        MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        unsigned blocks = (unsigned)((S.n + 255) / 256);
        double qw = S.q * S.w;
        int mixed = c.fp64 ? 0 : 1;
        if (c.d.shape_order == 1) k_rho<1><<<blocks, 256, 0, c.st>>>(c.g, qw, S.n, p64, pm, mixed, c.rho);
        else if (c.d.shape_order == 2) k_rho<2><<<blocks, 256, 0, c.st>>>(c.g, qw, S.n, p64, pm, mixed, c.rho);
        else k_rho<3><<<blocks, 256, 0, c.st>>>(c.g, qw, S.n, p64, pm, mixed, c.rho);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Kinetic energy sum_p w m (gamma - 1) dV (FP64).
// ---------------------------------------------------------------------------
__global__ void k_kinetic(int64_t n, Fp64Particles p64, MixedParticles pm, int mixed, double scale, double *out) {
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double u0, u1, u2;
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
__global__ void k_convert_in(int64_t n, int64_t off, const double *x, const double *y, const double *z,
                             const double *ux, const double *uy, const double *uz, double hx, double hy,
                             double hz, int nx, int ny, int nz, int mixed, Fp64Particles p64, MixedParticles pm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double in[3] = {x[t], y[t], z[t]};
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
        pm.ux[q] = (float)ux[t]; pm.uy[q] = (float)uy[t]; pm.uz[q] = (float)uz[t];
    } else {
        p64.x[q] = xi[0]; p64.y[q] = xi[1]; p64.z[q] = xi[2];
        p64.ux[q] = ux[t]; p64.uy[q] = uy[t]; p64.uz[q] = uz[t];
    }
}

cudaError_t launch_convert_in(Ctx &c, int s, int64_t off, int64_t n, const double *x, const double *y,
                              const double *z, const double *ux, const double *uy, const double *uz) {
    if (n == 0) return cudaSuccess;
    Species &S = c.sp[s];
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_convert_in<<<(unsigned)((n + 255) / 256), 256, 0, c.st>>>(n, off, x, y, z, ux, uy, uz, c.d.dx, c.d.dy, c.d.dz,
                                                               c.g.n[0], c.g.n[1], c.g.n[2], c.fp64 ? 0 : 1, p64, pm);
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
    Fp64Particles p64{S.x, S.y, S.z, S.ux, S.uy, S.uz};
    MixedParticles pm{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
    k_convert_out<<<(unsigned)((S.n + 255) / 256), 256, 0, c.st>>>(S.n, c.d.dx, c.d.dy, c.d.dz, c.fp64 ? 0 : 1,
                                                                   p64, pm, x, y, z, ux, uy, uz);
    ++c.nlaunch;
    return cudaGetLastError();
}

__global__ void k_check_finite(int64_t n, const double *a0, const double *a1, const double *a2, const double *a3,
                               const double *a4, const double *a5, int *flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s = a0[t] + a1[t] + a2[t] + a3[t] + a4[t] + a5[t];
    if (!isfinite(s) || !isfinite(a0[t]) || !isfinite(a1[t]) || !isfinite(a2[t]) || !isfinite(a3[t]) ||
        !isfinite(a4[t]) || !isfinite(a5[t]))
        atomicOr(flag, 1);
}

cudaError_t launch_check_finite(Ctx &c, int64_t n, const double *const *arrs, int narr, int *flag) {
    if (n == 0 || narr != 6) return cudaSuccess;
    k_check_finite<<<(unsigned)((n + 255) / 256), 256, 0, c.st>>>(n, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4],
                                                                 arrs[5], flag);
    ++c.nlaunch;
    return cudaGetLastError();
}

}  // namespace pp
