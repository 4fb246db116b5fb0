// pp_cells.cu -- the particle step of the mixed form on particles sorted by
// cell at the start of every step (Sec. III: the paper sorts the particle
// array by cell position in every step, between the current deposit and the
// field update, so that steps 1-3 run as one sweep that accumulates the
// current in small cache-resident buffers).
//
// One CTA per 8x8x8 tile of cells.  Because every particle of the tile's sorted
// range sits in the tile, the E/B window staged in shared memory is the tile
// plus the gather's reach only (12^3 nodes per component, copied by six TMA
// tensor copies that complete on an mbarrier whose wait is bounded in time),
// the current window the tile plus the deposit's reach (13^3 nodes), and the
// particles of one cell are consecutive in memory.  Per chunk of up to 4096
// particles of one species:
//
//  phase 1, one thread per particle (a warp on 32 consecutive particles, i.e.
//    one or two cells: the gather's shared loads are broadcasts): gather
//    (eq:pfields), push (Vay / Boris, optional radiative cooling), move; the
//    new cell, offset and momentum go straight back to the particle arrays
//    (coalesced); the old offset and the displacement are staged for the
//    deposit.  A particle whose support start changes on some axis (it
//    crosses a support boundary) is queued, with the axis and direction of
//    the change.
//  pieces: the chunk is cut into pieces of at most 8 consecutive particles
//    of one deposit group (the particles of one cell, and for even orders of
//    one octant of it, share their support start on every axis); the queue
//    (in chunk order) into crossing pieces of at most 8 consecutive entries
//    of one group that change their support start on the same single axis
//    in the same direction (so they share the union support: a cold beam's
//    particles of one cell that cross into the next one).
//  phase 2, the charge-conserving current (eq:cc1, eq:jj3, Esirkepov's
//    decomposition written as the 2nd-order current by a per-particle prefix
//    sum): one thread per (piece, component) sums the O (O+1)^2 site values
//    of its particles in registers and adds them to the tile's current
//    window with one shared atomic per site (about 48 x 3 per piece instead of
//    per particle); a crossing piece likewise over its union support (at most
//    (O+1)^3 sites per component); a particle that crosses on several axes
//    takes the general union form, with shared atomics per nonzero site.  A
//    warp's 32 items always share the component.
//
// The current window holds int32 fixed point (native shared integer atomics):
// each chunk takes its unit from its particles' motion so that no node can
// overflow, and after the chunk the nodes its cells reach are added into the
// FP32 mesh (one global atomic per nonzero node).  A piece's sum is FP32 in
// registers and is rounded to the unit once.
#include "pp_internal.cuh"
#include "pp_particle_common.cuh"
#include "pp_tma.cuh"

namespace pp {

namespace {

constexpr int kT = 8;                            // tile edge (cells)
constexpr int kTCells = kT * kT * kT;
constexpr int kRLo = 2, kRHi = 3;                // node reach below / above a cell (gather and deposit, O <= 3)
constexpr int kW = kT + kRLo + kRHi;             // 13 window nodes per axis
constexpr int kWVol = kW * kW * kW;              // words per window component
#ifndef PP_CELLS_THREADS
#define PP_CELLS_THREADS 512
#endif
constexpr int kCT = PP_CELLS_THREADS;            // threads per tile CTA
constexpr int kCW = kCT / 32;
// The E/B window the gather reads: nodes -2 .. 9 of the tile on each axis
// (a PCS support reaches two nodes either side of a particle's cell), one box
// of kWG^3 nodes per component copied by one TMA tensor copy (rows of 48
// bytes, a multiple of 16 as the copy requires), the six components kFComp
// words apart (128-byte aligned), then a 128-byte slot for the mbarrier the
// copies complete on.  The current window keeps kW nodes per axis: a particle
// that moves to the next cell deposits one node further up.
constexpr int kWG = kT + kRLo + 2;                             // 12
constexpr int kFComp = (kWG * kWG * kWG + 31) / 32 * 32;       // 1728 words
constexpr uint32_t kFBoxBytes = sizeof(float) * kWG * kWG * kWG;  // 6912 bytes per component
constexpr size_t kFieldBytes = sizeof(float) * 6 * kFComp + 128;
__device__ __forceinline__ int fi(int i, int j, int k) { return i + kWG * (j + kWG * k); }
// A staging wait that has not completed after this long gives up (ST_TIMEOUT).
constexpr uint64_t kStageWaitNs = 1000000000ull;
#ifndef PP_CELLS_CHUNK
#define PP_CELLS_CHUNK 4096
#endif
constexpr int kCC = PP_CELLS_CHUNK;              // particles staged per chunk
constexpr int kCPer = kCC / kCT;                 // phase-1 particles per thread per chunk
// Pieces of at most 8 particles: more register sums to add than with 16 or 32,
// but the deposit items spread evenly over the threads (64^3 thermal PCS:
// 2.60 ms at 8 or 12, 2.64 at 16, 2.92 at 32).
#ifndef PP_CELLS_PIECE
#define PP_CELLS_PIECE 8
#endif
constexpr int kPiece = PP_CELLS_PIECE;           // most particles per deposit piece
// Staged arrays hold one pad word per 16 particles: the lanes of a deposit warp
// read particles about one piece (16) apart, which unpadded would fall in two
// banks.
constexpr int kCS = kCC + kCC / 16;              // words per staged array
__device__ __forceinline__ int sp(int q) { return q + (q >> 4); }
// Group word of a staged particle: its deposit group (bits 0-11), its
// crossing signature (bits 12-14: 0 no support start changes; 1 + 2a + up for
// a change on axis a alone, up when it moves up; 7 for changes on several
// axes) and kSkip (not deposited by a piece of non-crossing particles).
constexpr uint16_t kSkip = 0x8000;
constexpr int kSigShift = 12;
constexpr uint16_t kGrpMask = 0x0fff, kSigMask = 0x7000;
static_assert(kCC % kCT == 0 && kCT % 32 == 0, "chunk must split evenly over the CTA");
static_assert(kCPer * kCW <= 1024, "piece-count table");
// counts (queue, -, pieces), box (6), totals (3); then four tables of
// per-(round, warp) counts and the crossing pieces per bucket (4)
constexpr int kMisc = 20 + 4 * kCPer * kCW;
// A crossing piece is stored as its first queue entry (12 bits) and its
// length - 1 (3 bits).
static_assert(kCC <= 4096 && kPiece <= 8, "crossing-piece word");
constexpr size_t kCellsSmem = kFieldBytes + sizeof(float) * (3 * kWVol + 6 * kCS) + sizeof(uint16_t) * (4 * kCC + 4) +
                              sizeof(int) * kMisc;
// The current window: an int32 fixed-point window whose unit each chunk takes
// from its particles' motion, flushed into the FP32 mesh per chunk; or, with
// PP_CELLS_FIXED=0, an FP32 window of shared FP32 atomics flushed once per
// tile.  Shared FP32 atomics measured about four times the shared-memory
// wavefronts of int32 ones here (64^3 thermal PCS: 4.67 against 2.51 ms).
#ifndef PP_CELLS_FIXED
#define PP_CELLS_FIXED 1
#endif
#if PP_CELLS_FIXED
using JT = int;
#else
using JT = float;
#endif
constexpr float kFixedRange = 1073741824.0f;    // 2^30
__device__ __forceinline__ void jadd(JT *p, float v) {
#if PP_CELLS_FIXED
    atomicAdd(p, __float2int_rn(v));
#else
    atomicAdd(p, v);
#endif
}
static_assert(kCellsSmem <= 227 * 1024, "tile CTA must fit the opt-in shared memory");

__device__ __forceinline__ int wi(int i, int j, int k) { return i + kW * (j + kW * k); }

// Gather accessor over the staged E/B window (frame = the particle's cell).
struct CellsFieldAcc {
    const float *Fw;
    int base;
    PP_IF_CHECKED(int wx = 0, wy = 0, wz = 0; int *st = nullptr; mutable int bad = 0;)
#ifdef PP_CHECKED
    __device__ __forceinline__ bool inside(int i, int j, int k) const {
        return wx + i >= 0 && wx + i < kWG && wy + j >= 0 && wy + j < kWG && wz + k >= 0 && wz + k < kWG;
    }
    __device__ ~CellsFieldAcc() {
        if (bad && st) atomicOr(st, ST_BOUNDS);
    }
#endif
    __device__ __forceinline__ float F(int kind, int comp, int i, int j, int k) const {
        PP_IF_CHECKED(if (!inside(i, j, k)) { bad = 1; return 0.0f; })
        return Fw[(kind * 3 + comp) * kFComp + base + fi(i, j, k)];
    }
};

// Current accessor over the FP32 shared window (frame = the particle's cell).
struct CellsCurrentAcc {
    JT *J;
    int base;
    PP_IF_CHECKED(int wx = 0, wy = 0, wz = 0; int *st = nullptr; mutable int bad = 0;)
#ifdef PP_CHECKED
    __device__ __forceinline__ bool inside(int i, int j, int k) const {
        return wx + i >= 0 && wx + i < kW && wy + j >= 0 && wy + j < kW && wz + k >= 0 && wz + k < kW;
    }
    __device__ ~CellsCurrentAcc() {
        if (bad && st) atomicOr(st, ST_BOUNDS);
    }
#endif
    __device__ __forceinline__ void addJ(int comp, int i, int j, int k, float v) const {
        PP_IF_CHECKED(if (!inside(i, j, k)) { bad = 1; return; })
        jadd(J + comp * kWVol + base + wi(i, j, k), v);
    }
};

struct CellsSpecies {
    MixedParticles p;            // read: slot i of the sorted order is p[perm[i]] (p[i] without perm)
    MixedParticles out;          // written: the new state of slot i, in the sorted order
    const int32_t *perm;         // pending sort permutation, or null
    int32_t *keys;               // written: the sort key of each slot's new state
    const int32_t *cell_start;   // per sort key, tile-major
    float qmdt;
    float kdt;                   // radiative cooling K / dt (0 = off)
    float jscale[3];             // -q w dx_a / dt
};

struct CellsArgs {
    CUtensorMap tmap[6];         // E_x, E_y, E_z, B_x, B_y, B_z: boxes of kWG^3 nodes
    Geom g;
    const float *E[3];
    const float *B[3];
    float *J[3];
    float dtdx[3];
    int nt[3];
    int ns;
    CellsSpecies sp[PP_MAX_SPECIES];
    int *status;
    int wall[3];                 // walls at 0 and wall[a] cells on axis a; 0 = periodic
    double esc;                  // open end: outgoing particles below x = esc cells leave; 0 = off
    int32_t dead_key;            // sort key of a particle that left: after every cell's keys
};

// Sort key of a particle in cell (x, y, z) with offsets o (the key of the cell
// sort: its 8^3 tile in tile order, its cell in the tile, the octant of the
// cell that holds it), or dead_key for a particle that left.
__device__ __forceinline__ int32_t sort_key(const CellsArgs &T, int32_t cw, const float (&o)[3]) {
    if (cw < 0) return T.dead_key;
    int x, y, z;
    unpack_cell(cw, x, y, z);
    const int tile = ((z / kT) * T.nt[1] + y / kT) * T.nt[0] + x / kT;
    const int cell = ((z % kT) * kT + y % kT) * kT + x % kT;
    const int oct = (o[0] >= 0.5f ? 1 : 0) | (o[1] >= 0.5f ? 2 : 0) | (o[2] >= 0.5f ? 4 : 0);
    return (tile * kTCells + cell) * kSubKeys + oct;
}

__device__ __forceinline__ void store(const CellsArgs &T, const CellsSpecies &S, int64_t i, int32_t cw,
                                      const float (&o)[3], const float (&u)[3]) {
    S.out.cell[i] = cw;
    S.out.ox[i] = o[0]; S.out.oy[i] = o[1]; S.out.oz[i] = o[2];
    S.out.ux[i] = u[0]; S.out.uy[i] = u[1]; S.out.uz[i] = u[2];
    S.keys[i] = sort_key(T, cw, o);
}

// Deposit group of a particle: its cell in the tile, and for even orders the
// octant of the cell it sits in (the support start on integer nodes is
// floor(xi - (O-1)/2), which for even O depends on which half of the cell
// holds xi).
template <int O>
__device__ __forceinline__ int group_of(int rx, int ry, int rz, const float (&xi)[3]) {
    const int cell = rx + kT * (ry + kT * rz);
    if constexpr (O % 2 == 0) {
        const int oct = (xi[0] >= 0.5f ? 1 : 0) | (xi[1] >= 0.5f ? 2 : 0) | (xi[2] >= 0.5f ? 4 : 0);
        return (cell << 3) | oct;
    } else {
        return cell;
    }
}

// Window coordinates of the group's cell and of its support start.
template <int O>
__device__ __forceinline__ void group_frame(int grp, int (&cw)[3], int (&lo)[3]) {
    const int cell = (O % 2 == 0) ? (grp >> 3) : grp;
    const int r[3] = {cell & (kT - 1), (cell / kT) & (kT - 1), cell / (kT * kT)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cw[d] = r[d] + kRLo;
        if constexpr (O % 2 == 0) lo[d] = cw[d] - (O - 2) / 2 - 1 + ((grp >> d) & 1);
        else lo[d] = cw[d] - (O - 1) / 2;
    }
}

// Component A of the current of the piece [s, e): the particles that cross no
// support boundary (flag clear) share the support start lo, so their
// O (O+1)^2 site values (those of deposit_esirkepov_inner, site by site) are
// summed in registers and added once.
template <int O, int A>
__device__ __forceinline__ void piece_current(JT *Jw, const float *s_o, const float *s_d, const uint16_t *s_grp,
                                              int s, int e, float jscale PP_IF_CHECKED(, int *st)) {
    constexpr int Bx = (A + 1) % 3, Cx = (A + 2) % 3;
    int cw[3], lo[3];
    group_frame<O>(s_grp[s] & kGrpMask, cw, lo);
    float acc[O][O + 1][O + 1];
#pragma unroll
    for (int m = 0; m < O; ++m)
#pragma unroll
        for (int mb = 0; mb <= O; ++mb)
#pragma unroll
            for (int mc = 0; mc <= O; ++mc) acc[m][mb][mc] = 0.0f;
#pragma unroll 1
    for (int q = s; q < e; ++q) {
        if (s_grp[q] & kSkip) continue;
        float S0[3][O + 1], DS[3][O + 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float x0 = s_o[d * kCS + sp(q)];
            const float x1 = x0 + s_d[d * kCS + sp(q)];
            float wo[O + 1], wn[O + 1];
            support<O, float>(x0, false, wo);
            support<O, float>(x1, false, wn);
#pragma unroll
            for (int m = 0; m <= O; ++m) {
                S0[d][m] = wo[m];
                DS[d][m] = wn[m] - wo[m];
            }
        }
        // prefix of dS along A (suffix form on the upper faces; the last face is 0)
        float C[O];
        float run = 0.0f;
#pragma unroll
        for (int m = 0; m < O; ++m) {
            if (2 * m < O + 1) {
                run += DS[A][m];
                C[m] = run * jscale;
            }
        }
        run = 0.0f;
#pragma unroll
        for (int m = O - 1; m >= 0; --m) {
            if (2 * m >= O + 1) {
                run -= DS[A][m + 1];
                C[m] = run * jscale;
            }
        }
#pragma unroll
        for (int mc = 0; mc <= O; ++mc) {
            const float p = S0[Cx][mc] + 0.5f * DS[Cx][mc];
            const float h = 0.5f * S0[Cx][mc] + (1.0f / 3.0f) * DS[Cx][mc];
#pragma unroll
            for (int mb = 0; mb <= O; ++mb) {
                const float Y = S0[Bx][mb] * p + DS[Bx][mb] * h;
#pragma unroll
                for (int m = 0; m < O; ++m) acc[m][mb][mc] += C[m] * Y;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < O; ++m)
#pragma unroll
        for (int mb = 0; mb <= O; ++mb)
#pragma unroll
            for (int mc = 0; mc <= O; ++mc) {
                int idx[3];
                idx[A] = lo[A] + m;
                idx[Bx] = lo[Bx] + mb;
                idx[Cx] = lo[Cx] + mc;
#ifdef PP_CHECKED
                if (idx[0] < 0 || idx[0] >= kW || idx[1] < 0 || idx[1] >= kW || idx[2] < 0 || idx[2] >= kW) {
                    atomicOr(st, ST_BOUNDS);
                    continue;
                }
#endif
                jadd(Jw + A * kWVol + wi(idx[0], idx[1], idx[2]), acc[m][mb][mc]);
            }
}

// Component A of the current of a particle whose support start moves on
// several axes: the general form on the union of its old and new supports
// (O + 2 nodes per axis).  Rare (a few particles per thousand even in a hot
// plasma), so kept out of line: the tile loop's code stays small enough for
// the instruction cache.
template <int O, int A>
__device__ __noinline__ void queued_current(JT *Jw, const float *s_o, const float *s_d, const uint16_t *s_grp,
                                               int q, float jscale PP_IF_CHECKED(, int *st)) {
    int cw[3], lo0[3];
    group_frame<O>(s_grp[q] & kGrpMask, cw, lo0);
    float xi0[3], xi1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xi0[d] = s_o[d * kCS + sp(q)];
        xi1[d] = xi0[d] + s_d[d * kCS + sp(q)];
    }
    CellsCurrentAcc acc{Jw, wi(cw[0], cw[1], cw[2])};
    PP_IF_CHECKED(acc.wx = cw[0]; acc.wy = cw[1]; acc.wz = cw[2]; acc.st = st;)
    float S0[3][O + 2], DS[3][O + 2];
    int lo[3];
    esirkepov_weights<O, float>(xi0, xi1, S0, DS, lo);
    esirkepov_component<O, float, A>(acc, S0, DS, lo, jscale);
}

// Component A of the current of a crossing piece: particles of one deposit
// group whose support start moves one node along axis XA alone, all in the
// same direction (up: to the next node), so that they share the union support
// (O + 2 nodes along XA, O + 1 along the others).  Their site values are those
// of the general union form (esirkepov_weights + esirkepov_component, site by
// site the same products; its sites that are zero for such a particle are
// left out here): NA faces along A (O + 1 when A is the crossing axis, else O,
// the last face being zero) times the union nodes across.  They are summed in
// registers over the piece and added once per site.  The work is written in
// axes rotated so that the crossing axis comes first (rotated axis r is axis
// (r + XA) mod 3, RA the rotated A), so that one body serves all three
// crossing axes.
template <int O, int RA>
__device__ __forceinline__ void cross_piece(JT *Jw, int A, int XA, const float *s_o, const float *s_d,
                                            const uint16_t *s_queue, int ks, int ke, int grp, bool up,
                                            float jscale PP_IF_CHECKED(, int *st)) {
    constexpr int RB = (RA + 1) % 3, RC = (RA + 2) % 3;
    constexpr int NA = (RA == 0) ? O + 1 : O;
    constexpr int NB = (RB == 0) ? O + 2 : O + 1;
    constexpr int NC = (RC == 0) ? O + 2 : O + 1;
    int cw[3], lo[3];
    group_frame<O>(grp, cw, lo);
    const int p[3] = {XA, XA == 2 ? 0 : XA + 1, XA == 0 ? 2 : XA - 1};   // physical axis of rotated axis r
    int lr[3], sr[3];   // support start and window stride per rotated axis
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        lr[r] = p[r] == 0 ? lo[0] : (p[r] == 1 ? lo[1] : lo[2]);
        sr[r] = p[r] == 0 ? 1 : (p[r] == 1 ? kW : kW * kW);
    }
    lr[0] -= up ? 0 : 1;   // union start along the crossing axis: the lower of the old and new starts
    float acc[NA][NB][NC];
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
        for (int mb = 0; mb < NB; ++mb)
#pragma unroll
            for (int mc = 0; mc < NC; ++mc) acc[m][mb][mc] = 0.0f;
#pragma unroll 1
    for (int e = ks; e < ke; ++e) {
        const int q = s_queue[e];
        float S0[3][O + 2], DS[3][O + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float x0 = s_o[p[r] * kCS + sp(q)];
            const float x1 = x0 + s_d[p[r] * kCS + sp(q)];
            float wo[O + 1], wn[O + 1];
            support<O, float>(x0, false, wo);
            support<O, float>(x1, false, wn);
            if (r == 0) {   // old weights from the union start (up) or one node above it
#pragma unroll
                for (int m = 0; m < O + 2; ++m) {
                    const float a0 = up ? (m <= O ? wo[m] : 0.0f) : (m >= 1 ? wo[m - 1] : 0.0f);
                    const float a1 = up ? (m >= 1 ? wn[m - 1] : 0.0f) : (m <= O ? wn[m] : 0.0f);
                    S0[r][m] = a0;
                    DS[r][m] = a1 - a0;
                }
            } else {
#pragma unroll
                for (int m = 0; m <= O; ++m) {
                    S0[r][m] = wo[m];
                    DS[r][m] = wn[m] - wo[m];
                }
                S0[r][O + 1] = 0.0f;
                DS[r][O + 1] = 0.0f;
            }
        }
        // prefix of dS along A on the lower faces, suffix on the upper ones
        float C[NA];
        float run = 0.0f;
#pragma unroll
        for (int m = 0; m < NA; ++m) {
            if (2 * m < O + 1) {
                run += DS[RA][m];
                C[m] = run * jscale;
            }
        }
        run = 0.0f;
#pragma unroll
        for (int m = NA - 1; m >= 0; --m) {
            if (2 * m >= O + 1) {
                run -= DS[RA][m + 1];
                C[m] = run * jscale;
            }
        }
#pragma unroll
        for (int mc = 0; mc < NC; ++mc) {
            const float pc = S0[RC][mc] + 0.5f * DS[RC][mc];
            const float hc = 0.5f * S0[RC][mc] + (1.0f / 3.0f) * DS[RC][mc];
#pragma unroll
            for (int mb = 0; mb < NB; ++mb) {
                const float Y = S0[RB][mb] * pc + DS[RB][mb] * hc;
#pragma unroll
                for (int m = 0; m < NA; ++m) acc[m][mb][mc] += C[m] * Y;
            }
        }
    }
    JT *J = Jw + A * kWVol;
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
        for (int mb = 0; mb < NB; ++mb)
#pragma unroll
            for (int mc = 0; mc < NC; ++mc) {
#ifdef PP_CHECKED
                if (lr[RA] + m < 0 || lr[RA] + m >= kW || lr[RB] + mb < 0 || lr[RB] + mb >= kW || lr[RC] + mc < 0 ||
                    lr[RC] + mc >= kW) {
                    atomicOr(st, ST_BOUNDS);
                    continue;
                }
#endif
                jadd(J + (lr[RA] + m) * sr[RA] + (lr[RB] + mb) * sr[RB] + (lr[RC] + mc) * sr[RC], acc[m][mb][mc]);
            }
}

// Component A of the current of the crossing piece [ks, ke) of the queue, of
// bucket xa: the crossing axis (cross_piece), or 3 for a single particle whose
// support start moves on several axes (the general union form).
template <int O>
__device__ __forceinline__ void xpiece_current(JT *Jw, int A, const float *s_o, const float *s_d,
                                               const uint16_t *s_grp, const uint16_t *s_queue, int ks, int ke, int xa,
                                               float jscale PP_IF_CHECKED(, int *st)) {
    if (xa == 3) {
        if (A == 0) queued_current<O, 0>(Jw, s_o, s_d, s_grp, s_queue[ks], jscale PP_IF_CHECKED(, st));
        else if (A == 1) queued_current<O, 1>(Jw, s_o, s_d, s_grp, s_queue[ks], jscale PP_IF_CHECKED(, st));
        else queued_current<O, 2>(Jw, s_o, s_d, s_grp, s_queue[ks], jscale PP_IF_CHECKED(, st));
        return;
    }
    const int g0 = s_grp[s_queue[ks]];
    const bool up = (((g0 & kSigMask) >> kSigShift) & 1) == 0;   // signature 1 + 2 xa + up
    const int grp = g0 & kGrpMask;
    const int ra = A >= xa ? A - xa : A - xa + 3;
    if (ra == 0) cross_piece<O, 0>(Jw, A, xa, s_o, s_d, s_queue, ks, ke, grp, up, jscale PP_IF_CHECKED(, st));
    else if (ra == 1) cross_piece<O, 1>(Jw, A, xa, s_o, s_d, s_queue, ks, ke, grp, up, jscale PP_IF_CHECKED(, st));
    else cross_piece<O, 2>(Jw, A, xa, s_o, s_d, s_queue, ks, ke, grp, up, jscale PP_IF_CHECKED(, st));
}

__device__ __forceinline__ unsigned lanemask_lt_() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan, in chunk order, of the per-(round, warp) counts
// c[0 .. kCPer kCW) by one warp; the total goes to *total.
__device__ __forceinline__ void scan_counts(int *c, int *total, int lane) {
    constexpr int kPerLane = (kCPer * kCW + 31) / 32;
    int v[kPerLane], sum = 0;
#pragma unroll
    for (int m = 0; m < kPerLane; ++m) {
        const int k = lane * kPerLane + m;
        v[m] = k < kCPer * kCW ? c[k] : 0;
        sum += v[m];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int run = incl - sum;
#pragma unroll
    for (int m = 0; m < kPerLane; ++m) {
        const int k = lane * kPerLane + m;
        if (k < kCPer * kCW) c[k] = run;
        run += v[m];
    }
    if (lane == 31) *total = incl;
}

// BND: walls (reflection) and the open end (escape); a separate instantiation
// so that periodic runs carry none of their tests.
// One tile of one run: the whole particle step of the tile's particles (all
// species), its current added into the run's mesh.  Called by every thread
// of the CTA; smem is the CTA's dynamic shared memory.
// Returns false when the CTA must stop: a staging wait ran out (here or in
// another CTA, ST_TIMEOUT).  phase: parity of the CTA's staging mbarrier, which
// the kernel initialised.  GMAPS: the tensor maps sit in global memory.
template <int O, int PUSH, bool BND, bool GMAPS>
__device__ __forceinline__ bool cells_tile(const CellsArgs &T, const int tile, float *smem, uint32_t &phase) {
    float *F = smem;
    uint64_t *bar = (uint64_t *)((char *)smem + kFieldBytes - 128);
    JT *Jw = (JT *)((char *)smem + kFieldBytes);
    float *s_o = (float *)(Jw + 3 * kWVol);   // 3 x kCS: offsets at t (frame of the cell)
    float *s_d = s_o + 3 * kCS;           // 3 x kCS: displacement of the step
    uint16_t *s_grp = (uint16_t *)(s_d + 3 * kCS);   // group word (deposit group, crossing, kSkip)
    uint16_t *s_piece = s_grp + kCC;                  // piece starts (+ the end)
    uint16_t *s_queue = s_piece + kCC + 2;            // crossing particles, in chunk order
    uint16_t *s_xpiece = s_queue + kCC;               // crossing pieces by bucket: first entry | (length - 1) << 12
    int *misc = (int *)(s_xpiece + kCC + 2);   // [0]: queue length; [2]: pieces;
                                               // [4..9]: fixed point: cell box of the chunk; [10..12]: sum |dxi|
    int *cnt = misc + 16;                 // starts per (round, warp); four tables
    int *qcnt = cnt + kCPer * kCW;        // crossing particles per (round, warp)
    int *xtot = cnt + 4 * kCPer * kCW;    // crossing pieces per bucket
    const Geom &g = T.g;
    const int tx = tile % T.nt[0], ty = (tile / T.nt[0]) % T.nt[1], tz = tile / (T.nt[0] * T.nt[1]);
    const int ox = tx * kT, oy = ty * kT, oz = tz * kT;
    const int wx = ox - kRLo, wy = oy - kRLo, wz = oz - kRLo;
    const int64_t key0 = (int64_t)tile * kTCells * kSubKeys, key1 = key0 + kTCells * kSubKeys;
    {   // a tile that holds no particle (the mirror half of a box between walls) stages nothing
        int held = 0;
        for (int s = 0; s < T.ns; ++s) held |= T.sp[s].cell_start[key1] - T.sp[s].cell_start[key0];
        if (!held) return true;
    }
    // ---- the E/B window by six TMA tensor copies (array coordinates of the
    // window's first node; the host checked that every tile's box lies inside
    // the padded arrays with an aligned x; rechecked here, uniformly, so that
    // no copy can start misaligned or outside)
    const int x0 = wx + g.G, y0 = wy + g.G, z0 = wz + g.G;
    if ((x0 & 3) || x0 < 0 || y0 < 0 || z0 < 0 || x0 + kWG > g.P[0] || y0 + kWG > g.P[1] || z0 + kWG > g.P[2]) {
        if (threadIdx.x == 0) atomicOr(T.status, ST_BOUNDS);
        return true;
    }
    if (threadIdx.x == 0) {
        // a CTA whose wait ran out stops the others at their next tile
        misc[3] = (*(volatile int *)T.status & ST_TIMEOUT) != 0;
        if (misc[3]) {
            mbar_arrive(bar);
        } else {
            fence_proxy_async_smem();   // the previous tile's reads of F come before the copies' writes
            mbar_arrive_expect(bar, 6 * kFBoxBytes);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if (GMAPS) fence_tensormap_acquire(&T.tmap[c]);
                tma_load_3d(F + c * kFComp, &T.tmap[c], x0, y0, z0, bar);
            }
        }
    }
    for (int idx = threadIdx.x; idx < 3 * kWVol; idx += kCT) Jw[idx] = 0;
    if (!cta_wait_bounded(bar, phase, kStageWaitNs, T.status)) return false;
    phase ^= 1;
    if (misc[3]) return false;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < T.ns; ++s) {
        const CellsSpecies &S = T.sp[s];
        const int tb = S.cell_start[key0], te = S.cell_start[key1];
        for (int cb = tb; cb < te; cb += kCC) {
            const int cn = min(kCC, te - cb);
#if PP_CELLS_FIXED
            float sum[3] = {0.0f, 0.0f, 0.0f};
            int blo[3] = {kT, kT, kT}, bhi[3] = {-1, -1, -1};
#endif
            // ---- phase 1: gather, push, move; write back; stage the deposit
            // the particle of the next round is fetched (through the pending
            // permutation) before the current one is computed, so that its
            // dependent global loads overlap the gather
            int32_t n_cw = 0;
            float n_o[3] = {0.0f, 0.0f, 0.0f}, n_u[3] = {0.0f, 0.0f, 0.0f};
            auto fetch = [&](int qf) {
                if (qf >= cn) return;
                const int64_t i = (int64_t)cb + qf;
                const int64_t src = S.perm ? (int64_t)S.perm[i] : i;
                n_cw = S.p.cell[src];
                n_o[0] = S.p.ox[src]; n_o[1] = S.p.oy[src]; n_o[2] = S.p.oz[src];
                n_u[0] = S.p.ux[src]; n_u[1] = S.p.uy[src]; n_u[2] = S.p.uz[src];
            };
            fetch(threadIdx.x);
#pragma unroll 1
            for (int r = 0; r < kCPer; ++r) {
                const int q = r * kCT + threadIdx.x;
                if (q >= cn) break;
                const int64_t idx = (int64_t)cb + q;
                const int32_t cw0 = n_cw;
                float xi0[3] = {n_o[0], n_o[1], n_o[2]};
                float u[3] = {n_u[0], n_u[1], n_u[2]};
                fetch(q + kCT);
                int cx, cy, cz;
                unpack_cell(cw0, cx, cy, cz);
                const int rx = cx - ox, ry = cy - oy, rz = cz - oz;
                if ((unsigned)rx >= (unsigned)kT || (unsigned)ry >= (unsigned)kT || (unsigned)rz >= (unsigned)kT) {
                    // not in its sorted tile: cannot happen after a sort; left unmoved and flagged
                    atomicOr(T.status, ST_RANGE);
                    s_grp[q] = kSkip;
                    store(T, S, idx, cw0, xi0, u);
                    continue;
                }
                const float u0[3] = {u[0], u[1], u[2]};
                const int grp = group_of<O>(rx, ry, rz, xi0);
                if (S.qmdt != 0.0f) {   // uniform: no kick, no force
                    float E[3], B[3];
                    CellsFieldAcc facc{F, fi(rx + kRLo, ry + kRLo, rz + kRLo)};
                    PP_IF_CHECKED(facc.wx = rx + kRLo; facc.wy = ry + kRLo; facc.wz = rz + kRLo; facc.st = T.status;)
                    gather_EB<O, float>(facc, xi0, E, B);
                    push_particle<PUSH, float>(S.qmdt, S.kdt, E, B, u);
                }
                const float gi = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                float dx[3], xi1[3];
                bool ok = true;
                int ncross = 0, xa = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    dx[d] = T.dtdx[d] * u[d] * gi;
                    xi1[d] = xi0[d] + dx[d];
                    ok = ok && (fabsf(dx[d]) < 1.0f);
                    if (floorf(xi0[d] - 0.5f * (O - 1)) != floorf(xi1[d] - 0.5f * (O - 1))) {
                        ++ncross;
                        xa = d;
                    }
                }
                if (!ok) {   // leave the particle unchanged and flag the step
                    atomicOr(T.status, isfinite(u[0] + u[1] + u[2]) ? ST_CFL : ST_NAN);
                    s_grp[q] = (uint16_t)(grp | kSkip);
                    store(T, S, idx, cw0, xi0, u0);
                    continue;
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    s_o[d * kCS + sp(q)] = xi0[d];
                    s_d[d * kCS + sp(q)] = dx[d];
                }
#if PP_CELLS_FIXED
                sum[0] += fabsf(dx[0]); sum[1] += fabsf(dx[1]); sum[2] += fabsf(dx[2]);
                blo[0] = min(blo[0], rx); blo[1] = min(blo[1], ry); blo[2] = min(blo[2], rz);
                bhi[0] = max(bhi[0], rx); bhi[1] = max(bhi[1], ry); bhi[2] = max(bhi[2], rz);
#endif
                // crossing signature: the axis and direction of a support start
                // that moves on one axis alone, 7 when it moves on several
                const int sig = ncross == 0 ? 0 : (ncross == 1 ? 1 + 2 * xa + (dx[xa] > 0.0f ? 1 : 0) : 7);
                s_grp[q] = (uint16_t)(grp | (sig << kSigShift) | (ncross ? kSkip : 0));
                // the new state, written to the slot (the deposit reads the staged copy)
                int ncx = cx, ncy = cy, ncz = cz;
                rebin(xi1[0], ncx, g.n[0]);
                rebin(xi1[1], ncy, g.n[1]);
                rebin(xi1[2], ncz, g.n[2]);
                int32_t cwd;
                if constexpr (BND) {
                    reflect(ncx, xi1[0], u[0], T.wall[0]);
                    reflect(ncy, xi1[1], u[1], T.wall[1]);
                    reflect(ncz, xi1[2], u[2], T.wall[2]);
                    cwd = pack_cell(ncx, ncy, ncz);
                    if (T.esc > 0.0 && (double)ncx + (double)xi1[0] < T.esc && u[0] < 0.0f) cwd |= kDeadBit;
                } else {
                    cwd = pack_cell(ncx, ncy, ncz);
                }
                store(T, S, idx, cwd, xi1, u);
            }
#if PP_CELLS_FIXED
            if (threadIdx.x < 3) {   // previous chunk's values were last read before the barrier above
                misc[4 + threadIdx.x] = kT;
                misc[7 + threadIdx.x] = -1;
                ((float *)misc)[10 + threadIdx.x] = 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float sd = sum[d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
                const int l = __reduce_min_sync(0xffffffffu, blo[d]), h = __reduce_max_sync(0xffffffffu, bhi[d]);
                if (lane == 0) {
                    atomicAdd((float *)misc + 10 + d, sd);
                    atomicMin(misc + 4 + d, l);
                    atomicMax(misc + 7 + d, h);
                }
            }
#endif
            __syncthreads();
            // ---- pieces of non-crossing particles: starts at a group change and
            // every kPiece-th particle; crossing particles into the queue, in chunk
            // order (both by ballots and a scan of the per-(round, warp) counts)
            unsigned ball[kCPer], qball[kCPer];
#pragma unroll
            for (int r = 0; r < kCPer; ++r) {
                const int q = r * kCT + threadIdx.x;
                bool st = false, cr = false;
                if (q < cn) {
                    const int gq = s_grp[q];
                    st = q % kPiece == 0 || ((gq ^ s_grp[q - 1]) & kGrpMask) != 0;
                    cr = (gq & kSigMask) != 0;
                }
                ball[r] = __ballot_sync(0xffffffffu, st);
                qball[r] = __ballot_sync(0xffffffffu, cr);
                if (lane == 0) {
                    cnt[r * kCW + warp] = __popc(ball[r]);
                    qcnt[r * kCW + warp] = __popc(qball[r]);
                }
            }
            __syncthreads();
            if (warp == 0) scan_counts(cnt, misc + 2, lane);
            else if (warp == 1) scan_counts(qcnt, misc + 0, lane);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kCPer; ++r) {
                const int q = r * kCT + threadIdx.x;
                const unsigned below = lanemask_lt_();
                if (ball[r] & (1u << lane)) s_piece[cnt[r * kCW + warp] + __popc(ball[r] & below)] = (uint16_t)q;
                if (qball[r] & (1u << lane)) s_queue[qcnt[r * kCW + warp] + __popc(qball[r] & below)] = (uint16_t)q;
            }
            if (threadIdx.x == 0) s_piece[misc[2]] = (uint16_t)cn;
            __syncthreads();
            // ---- crossing pieces over the queue: starts at a change of group or
            // crossing, at a particle crossing on several axes and after one, and
            // every kPiece-th entry.  They are listed by bucket (the crossing axis,
            // or 3 for several axes), so that the 32 items of a warp take one form.
            const int nq = misc[0];
            auto xstart = [&](int k) {
                const int gk = s_grp[s_queue[k]];
                if (k % kPiece == 0 || (gk & kSigMask) == kSigMask) return true;
                const int gp = s_grp[s_queue[k - 1]];
                return (gp & kSigMask) == kSigMask || ((gk ^ gp) & (kGrpMask | kSigMask)) != 0;
            };
            int xflag = 0;   // per round: bit 2 start, bits 0-1 bucket
#pragma unroll
            for (int r = 0; r < kCPer; ++r) {
                const int k = r * kCT + threadIdx.x;
                int f = 0;
                if (k < nq && xstart(k)) f = 4 | ((((s_grp[s_queue[k]] & kSigMask) >> kSigShift) - 1) >> 1);
                xflag |= f << (3 * r);
#pragma unroll
                for (int bk = 0; bk < 4; ++bk) {
                    const unsigned m = __ballot_sync(0xffffffffu, f == (4 | bk));
                    if (lane == 0) cnt[bk * kCPer * kCW + r * kCW + warp] = __popc(m);
                }
            }
            __syncthreads();
            if (warp < 4) scan_counts(cnt + warp * kCPer * kCW, xtot + warp, lane);
            __syncthreads();
            const int xb1 = xtot[0], xb2 = xb1 + xtot[1], xb3 = xb2 + xtot[2];
#pragma unroll
            for (int r = 0; r < kCPer; ++r) {
                const int k = r * kCT + threadIdx.x;
                const int f = (xflag >> (3 * r)) & 7;
#pragma unroll
                for (int bk = 0; bk < 4; ++bk) {
                    const unsigned m = __ballot_sync(0xffffffffu, f == (4 | bk));
                    if (f == (4 | bk)) {
                        int e = k + 1;
                        while (e < nq && e % kPiece != 0 && !xstart(e)) ++e;
                        const int base = bk == 0 ? 0 : (bk == 1 ? xb1 : (bk == 2 ? xb2 : xb3));
                        s_xpiece[base + cnt[bk * kCPer * kCW + r * kCW + warp] + __popc(m & lanemask_lt_())] =
                            (uint16_t)(k | ((e - k - 1) << 12));
                    }
                }
            }
            __syncthreads();
            // ---- phase 2: current of the pieces, then of the crossing pieces; items in
            // blocks of 96 = 3 components x 32, so that a warp's items share the component
            const int np = misc[2];
            const int nblk = (np + 31) >> 5;
            // crossing pieces per bucket, their blocks of 32 (scalars: an array
            // indexed by the bucket would live in local memory)
            const int xn0 = xtot[0], xn1 = xtot[1], xn2 = xtot[2], xn3 = xtot[3];
            const int xk0 = (xn0 + 31) >> 5, xk1 = (xn1 + 31) >> 5, xk2 = (xn2 + 31) >> 5, xk3 = (xn3 + 31) >> 5;
            // current scale: -q w dx_a / dt, times the chunk's fixed-point unit; no
            // node can receive more than K_O |jscale_a| sum_p (|dxi_a| + 1e-6) from
            // the chunk (|C Y| <= K_O |dxi_a|, fixed_point_cy_bound), kept below 2^30
            // units; a piece or crossing piece converts its register sum once, so
            // a node collects at most one rounding half per piece, per crossing
            // piece and per particle crossing on several axes
            float jsc[3], unit[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
#if PP_CELLS_FIXED
                const float bound = fixed_point_cy_bound<O>() * fabsf(S.jscale[d]) *
                                    (((float *)misc)[10 + d] + 1e-6f * (float)cn) * 1.001f;
                unit[d] = bound > 0.0f ? kFixedRange / bound : 0.0f;
#else
                unit[d] = 1.0f;
#endif
                jsc[d] = S.jscale[d] * unit[d];
            }
            const int nitems = (nblk + xk0 + xk1 + xk2 + xk3) * 96;
#pragma unroll 1
            for (int it = threadIdx.x; it < nitems; it += kCT) {
                const int blk = it / 96, rr = it - blk * 96, comp = rr >> 5, j = rr & 31;
                // lane j of item block b takes piece (crossing piece) j * blocks + b:
                // consecutive pieces often share a cell, so lanes on consecutive
                // pieces would add to the same words
                if (blk < nblk) {
                    const int p = j * nblk + blk;
                    if (p >= np) continue;
                    const int ps = s_piece[p], pe = s_piece[p + 1];
                    if (comp == 0) piece_current<O, 0>(Jw, s_o, s_d, s_grp, ps, pe, jsc[0] PP_IF_CHECKED(, T.status));
                    else if (comp == 1) piece_current<O, 1>(Jw, s_o, s_d, s_grp, ps, pe, jsc[1] PP_IF_CHECKED(, T.status));
                    else piece_current<O, 2>(Jw, s_o, s_d, s_grp, ps, pe, jsc[2] PP_IF_CHECKED(, T.status));
                } else {   // crossing pieces: the block's bucket, then lane j's piece in it
                    int bk, lb = blk - nblk, nk, nn, base;
                    if (lb < xk0) {
                        bk = 0; nk = xk0; nn = xn0; base = 0;
                    } else if ((lb -= xk0) < xk1) {
                        bk = 1; nk = xk1; nn = xn1; base = xn0;
                    } else if ((lb -= xk1) < xk2) {
                        bk = 2; nk = xk2; nn = xn2; base = xn0 + xn1;
                    } else {
                        lb -= xk2;
                        bk = 3; nk = xk3; nn = xn3; base = xn0 + xn1 + xn2;
                    }
                    const int k = j * nk + lb;
                    if (k >= nn) continue;
                    const int v = s_xpiece[base + k];
                    const int ks = v & 0xfff, ke = ks + (v >> 12) + 1;
                    const float js = comp == 0 ? jsc[0] : (comp == 1 ? jsc[1] : jsc[2]);
                    xpiece_current<O>(Jw, comp, s_o, s_d, s_grp, s_queue, ks, ke, bk, js PP_IF_CHECKED(, T.status));
                }
            }
            __syncthreads();
#if PP_CELLS_FIXED
            {   // the window nodes the chunk's cells reach, into the FP32 mesh (and cleared)
                const int x0 = misc[4], y0 = misc[5], z0 = misc[6];
                if (misc[7] >= x0) {
                    const int ex = misc[7] - x0 + kRLo + kRHi + 1, ey = misc[8] - y0 + kRLo + kRHi + 1,
                              ez = misc[9] - z0 + kRLo + kRHi + 1;
                    const int vol = ex * ey * ez;
                    for (int idx = threadIdx.x; idx < 3 * vol; idx += kCT) {
                        const int comp = idx / vol, r = idx - comp * vol;
                        const int i = x0 + r % ex, j = y0 + (r / ex) % ey, k = z0 + r / (ex * ey);
                        JT *w = Jw + comp * kWVol + wi(i, j, k);
                        const int iv = *w;
                        if (iv == 0) continue;
                        *w = 0;
                        atomicAdd(T.J[comp] + g.at(wx + i, wy + j, wz + k), (float)iv / unit[comp]);
                    }
                }
                __syncthreads();
            }
#endif
        }
    }
#if !PP_CELLS_FIXED
    // ---- the tile's current, once into the FP32 mesh
    for (int idx = threadIdx.x; idx < 3 * kWVol; idx += kCT) {
        const float v = Jw[idx];
        if (v == 0.0f) continue;
        const int comp = idx / kWVol, r = idx - comp * kWVol;
        const int i = r % kW, j = (r / kW) % kW, k = r / (kW * kW);
        atomicAdd(T.J[comp] + g.at(wx + i, wy + j, wz + k), v);
    }
#endif
    return true;
}

// Dynamic shared memory starts 128-byte aligned (the TMA destinations); the
// kernels check it and stop (ST_BOUNDS) otherwise.
__device__ __forceinline__ bool smem_aligned(const float *smem, int *status) {
    if ((smem_addr(smem) & 127) == 0) return true;
    if (threadIdx.x == 0) atomicOr(status, ST_BOUNDS);
    return false;
}

template <int O, int PUSH, bool BND>
__global__ void __launch_bounds__(kCT, 1) k_particles_cells(const __grid_constant__ CellsArgs T) {
    extern __shared__ __align__(128) float smem[];
    if (!smem_aligned(smem, T.status)) return;
    uint64_t *bar = (uint64_t *)((char *)smem + kFieldBytes - 128);
    if (threadIdx.x == 0) mbar_init(bar);
    __syncthreads();
    uint32_t phase = 0;
    cells_tile<O, PUSH, BND, false>(T, blockIdx.x, smem, phase);
}

// Batched form: the tiles of many runs as (run, tile) work items, taken in
// order by persistent CTAs from a device counter (the items come sorted by
// run size, largest first, so that the last items are short).  Every run's
// arguments, tensor maps included, sit in device memory.
template <int O, int PUSH, bool BND>
__global__ void __launch_bounds__(kCT, 1) k_particles_cells_multi(const CellsArgs *args, const int2 *items,
                                                                 int nitems, int *next, int *status) {
    extern __shared__ __align__(128) float smem[];
    if (!smem_aligned(smem, status)) return;
    uint64_t *bar = (uint64_t *)((char *)smem + kFieldBytes - 128);
    int *item = (int *)(bar + 2);
    if (threadIdx.x == 0) mbar_init(bar);
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) *item = atomicAdd(next, 1);
        __syncthreads();
        const int w = *item;
        __syncthreads();   // every thread has read it before thread 0 takes the next
        if (w >= nitems) return;
        const int2 it = items[w];
        if (!cells_tile<O, PUSH, BND, true>(args[it.x], it.y, smem, phase)) return;
        __syncthreads();
    }
}

}  // namespace

// Besides the tile shape: every tile's TMA box starts at an x that is a
// multiple of 4 nodes (G - kRLo is, and tile origins are multiples of 8) and
// ends inside the padded row (G >= kWG - kT - kRLo), with rows of a multiple
// of 16 bytes.
bool cells_supported(const Ctx &c) {
    if (c.fp64 || c.current_mode != PP_CURRENT_CONSERVING || c.g.G < kRLo || c.g.G < kRHi) return false;
    if ((c.g.G - kRLo) % 4 != 0 || c.g.G < kWG - kT - kRLo || c.g.P[0] % 4 != 0) return false;
    for (int a = 0; a < 3; ++a)
        if (c.g.n[a] % kT != 0 || c.tile[a] != kT) return false;
    return true;
}

// The argument block of one context, with the tensor maps of its E and B
// arrays; any = false when no species holds particles.
static cudaError_t cells_args(const Ctx &c, CellsArgs &T, bool &any) {
    any = false;
    T.g = c.g;
    const double h[3] = {c.d.dx, c.d.dy, c.d.dz};
    for (int d = 0; d < 3; ++d) {
        T.E[d] = (const float *)c.E[d];
        T.B[d] = (const float *)c.B[d];
        T.J[d] = (float *)c.J[d];
        T.dtdx[d] = (float)(c.drift_dt / h[d]);
        T.nt[d] = c.ntile[d];
    }
    const int box[3] = {kWG, kWG, kWG};
    for (int comp = 0; comp < 6; ++comp) {
        cudaError_t e = encode_box_map(&T.tmap[comp], comp < 3 ? T.E[comp] : T.B[comp - 3], c.g.P, box);
        if (e != cudaSuccess) return e;
    }
    T.ns = 0;
    for (int s = 0; s < c.nspecies; ++s) {
        const Species &S = c.sp[s];
        if (S.n == 0) continue;
        CellsSpecies &t = T.sp[T.ns++];
        t.p = MixedParticles{S.cell, S.ox, S.oy, S.oz, S.fux, S.fuy, S.fuz};
        int32_t *c2 = (int32_t *)S.alt;
        float *f2 = (float *)(c2 + S.cap);
        t.out = MixedParticles{c2, f2, f2 + S.cap, f2 + 2 * S.cap, f2 + 3 * S.cap, f2 + 4 * S.cap, f2 + 5 * S.cap};
        t.perm = S.perm_pending ? S.perm : nullptr;
        t.keys = S.keys;
        t.cell_start = S.cell_start;
        t.qmdt = (float)(S.q * c.kick_dt / S.m);
        t.kdt = (float)(c.kick_dt != 0.0 ? S.rad / c.kick_dt : 0.0);
        for (int d = 0; d < 3; ++d) t.jscale[d] = (float)(-S.q * S.w * h[d] / c.drift_dt);
    }
    T.status = c.d_status;
    for (int d = 0; d < 3; ++d) T.wall[d] = c.wall[d];
    T.esc = c.escape_now;
    T.dead_key = (int32_t)c.nkeys;
    any = T.ns > 0;
    return cudaSuccess;
}

static bool cells_ready(const Ctx &c) {
    for (int s = 0; s < c.nspecies; ++s)
        if (c.sp[s].n > 0 && !c.sp[s].fresh) return false;
    return true;
}

// After the launch: every slot of the sorted order holds its particle's new
// state in the other buffer, with its next sort key.
static void cells_after(Ctx &c) {
    for (int s = 0; s < c.nspecies; ++s) {
        Species &S = c.sp[s];
        if (S.n == 0) continue;
        void *old = S.buf;
        S.buf = S.alt;
        S.alt = old;
        S.bind(false);
        S.perm_pending = false;
        S.keys_valid = true;
    }
}

template <class K>
static cudaError_t smem_attr(K kernel, unsigned long long &done) {
    return ensure_smem_attr(kernel, (int)kCellsSmem, done);
}

// All species in one launch; every species with particles must have been
// sorted since its particles last moved (Species::fresh).
cudaError_t launch_particles_cells(Ctx &c) {
    if (!cells_supported(c)) return cudaErrorInvalidConfiguration;
    if (!cells_ready(c)) return cudaErrorInvalidValue;
    CellsArgs T;
    bool any = false;
    cudaError_t ea = cells_args(c, T, any);
    if (ea != cudaSuccess || !any) return ea;
    const unsigned blocks = (unsigned)(c.ntile[0] * c.ntile[1] * c.ntile[2]);
    const int o = c.d.shape_order, pu = c.d.pusher;
    const bool bnd = c.any_wall();
    static unsigned long long attr_done[2][2][4] = {};
#define PP_CB(O, PU, BD)                                                                                     \
    do {                                                                                                     \
        cudaError_t e_ = smem_attr(k_particles_cells<O, PU, BD>, attr_done[BD][PU][O]);                      \
        if (e_ != cudaSuccess) return e_;                                                                    \
        k_particles_cells<O, PU, BD><<<blocks, kCT, kCellsSmem, c.st>>>(T);                                  \
    } while (0)
#define PP_C(O, PU)                                                                                          \
    do {                                                                                                     \
        if (bnd) PP_CB(O, PU, true); else PP_CB(O, PU, false);                                               \
    } while (0)
    if (pu == PP_BORIS) {
        if (o == 1) PP_C(1, PP_BORIS); else if (o == 2) PP_C(2, PP_BORIS); else PP_C(3, PP_BORIS);
    } else {
        if (o == 1) PP_C(1, PP_VAY); else if (o == 2) PP_C(2, PP_VAY); else PP_C(3, PP_VAY);
    }
#undef PP_C
#undef PP_CB
    ++c.nlaunch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cells_after(c);
    return cudaSuccess;
}

size_t cells_args_bytes() { return sizeof(CellsArgs); }

int cells_batch_key(const Ctx &c) { return c.d.shape_order * 4 + c.d.pusher * 2 + (c.any_wall() ? 1 : 0); }

// The tiles of n contexts with one cells_batch_key in one persistent launch of
// nsm CTAs on st.  host_args / host_items: pinned host memory of at least
// n * cells_args_bytes() and (sum of tiles) * 8 bytes, copied to the device
// scratch on st (the caller keeps them unchanged until the copy has run).
cudaError_t launch_particles_cells_batch(Ctx *const *ctxs, int n, cudaStream_t st, CellsBatchScratch &scr,
                                         void *host_args, void *host_items, int nsm) {
    if (n <= 0) return cudaSuccess;
    CellsArgs *A = (CellsArgs *)host_args;
    int2 *items = (int2 *)host_items;
    // runs with particles, largest first: their tiles become the first items
    int order[4096], m = 0;
    for (int k = 0; k < n && m < 4096; ++k) {
        Ctx &c = *ctxs[k];
        if (!cells_supported(c) || !cells_ready(c)) return cudaErrorInvalidValue;
        bool any = false;
        cudaError_t ea = cells_args(c, A[m], any);
        if (ea != cudaSuccess) return ea;
        if (any) order[m++] = k;
    }
    int64_t ntot = 0;
    for (int a = 0; a < m; ++a) {   // insertion sort by tile count, descending
        for (int b = a; b > 0; --b) {
            const Ctx &x = *ctxs[order[b]], &y = *ctxs[order[b - 1]];
            const int64_t tx = (int64_t)x.ntile[0] * x.ntile[1] * x.ntile[2];
            const int64_t ty = (int64_t)y.ntile[0] * y.ntile[1] * y.ntile[2];
            if (tx <= ty) break;
            const int t = order[b]; order[b] = order[b - 1]; order[b - 1] = t;
            CellsArgs u = A[b]; A[b] = A[b - 1]; A[b - 1] = u;
        }
    }
    for (int a = 0; a < m; ++a) {
        const Ctx &c = *ctxs[order[a]];
        const int tiles = c.ntile[0] * c.ntile[1] * c.ntile[2];
        for (int t = 0; t < tiles; ++t) items[ntot++] = make_int2(a, t);
    }
    if (m == 0) return cudaSuccess;
    const size_t abytes = sizeof(CellsArgs) * (size_t)m, ibytes = sizeof(int2) * (size_t)ntot;
    if (abytes > scr.args_cap || ibytes > scr.items_cap) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemcpyAsync(scr.args, A, abytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scr.items, items, ibytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scr.next, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const Ctx &c0 = *ctxs[order[0]];
    const int o = c0.d.shape_order, pu = c0.d.pusher;
    const bool bnd = c0.any_wall();
    const unsigned grid = (unsigned)(nsm < ntot ? nsm : ntot);
    static unsigned long long attr_done[2][2][4] = {};
#define PP_MB(O, PU, BD)                                                                                     \
    do {                                                                                                     \
        cudaError_t e_ = smem_attr(k_particles_cells_multi<O, PU, BD>, attr_done[BD][PU][O]);                \
        if (e_ != cudaSuccess) return e_;                                                                    \
        k_particles_cells_multi<O, PU, BD><<<grid, kCT, kCellsSmem, st>>>(                                   \
            (const CellsArgs *)scr.args, (const int2 *)scr.items, (int)ntot, scr.next, c0.d_status);         \
    } while (0)
#define PP_M(O, PU)                                                                                          \
    do {                                                                                                     \
        if (bnd) PP_MB(O, PU, true); else PP_MB(O, PU, false);                                               \
    } while (0)
    if (pu == PP_BORIS) {
        if (o == 1) PP_M(1, PP_BORIS); else if (o == 2) PP_M(2, PP_BORIS); else PP_M(3, PP_BORIS);
    } else {
        if (o == 1) PP_M(1, PP_VAY); else if (o == 2) PP_M(2, PP_VAY); else PP_M(3, PP_VAY);
    }
#undef PP_M
#undef PP_MB
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int a = 0; a < m; ++a) {
        Ctx &c = *ctxs[order[a]];
        ++c.nlaunch;
        cells_after(c);
    }
    return cudaSuccess;
}

}  // namespace pp
