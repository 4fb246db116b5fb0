// pp_internal.cuh -- shared declarations of the GB300 Photon-Plasma library.
//
// Device-side building blocks of the particle step (Sec. II weight functions,
// Sec. III pushers and charge-conserving deposit) and the context structure
// behind the C ABI of include/pp.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pp.h"

namespace pp {

// ---------------------------------------------------------------------------
// Mesh geometry: every mesh array is padded by G ghost layers per side,
// x fastest.  Interior index (i,j,k) in [0,n) maps to the padded offset below.
// ---------------------------------------------------------------------------
constexpr int kSubKeys = 8;  // sort sub-keys per cell: the octant of the particle inside it
// Ghost layers per side: 5 cover the deposit reach of a particle sorted up to
// two cells outside its tile plus the PCS support; the sixth makes the padded
// row (n + 12 nodes) a multiple of 16 bytes in FP32 for every n that is a
// multiple of 8, as the TMA tensor maps of the per-step kernel require.
constexpr int kGhost = 6;

struct Geom {
    int n[3];     // interior cells
    int P[3];     // padded extents n + 2G
    int G;
    __host__ __device__ __forceinline__ int64_t at(int i, int j, int k) const {
        return ((int64_t)(k + G) * P[1] + (j + G)) * P[0] + (i + G);
    }
    __host__ __device__ __forceinline__ int64_t padded_size() const { return (int64_t)P[0] * P[1] * P[2]; }
    __host__ __device__ __forceinline__ int64_t cells() const { return (int64_t)n[0] * n[1] * n[2]; }
};

// A particle that left the box (through an open end or the top layer of a
// sliding window) stays in its slot until the next sort drops it: the mixed
// form sets the sign bit of its packed cell, the FP64 form a negative x.
constexpr int32_t kDeadBit = (int32_t)0x80000000u;
constexpr double kDeadX = -1.0;

// Wrap an index that lies within a few periods of [0, n).
__host__ __device__ __forceinline__ int wrap(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// Device status bits (collected into one word, mapped to PP_* on the host).
enum : int { ST_NAN = 1, ST_CFL = 2, ST_NOCONV = 4, ST_RANGE = 8, ST_BOUNDS = 16, ST_TIMEOUT = 32 };

// Checked build (-DPP_CHECKED): the particle kernels test every mesh and
// shared-memory index against its array; a violation sets ST_BOUNDS in the
// status word and the access is skipped (a read returns 0), with no trap.
#ifdef PP_CHECKED
#define PP_IF_CHECKED(...) __VA_ARGS__
#else
#define PP_IF_CHECKED(...)
#endif

// ---------------------------------------------------------------------------
// B-spline weights of order O (Sec. II, W^1..W^3) written in the fractional
// coordinate f in [0,1) of the first support node: node i0+m has weight w[m].
// ---------------------------------------------------------------------------
template <int O, typename R>
__device__ __forceinline__ void bspline(R f, R (&w)[O + 1]) {
    if constexpr (O == 1) {
        w[0] = R(1) - f;
        w[1] = f;
    } else if constexpr (O == 2) {
        R g = R(1) - f;
        R h = f - R(0.5);
        w[0] = R(0.5) * g * g;
        w[1] = R(0.75) - h * h;
        w[2] = R(0.5) * f * f;
    } else {
        R g = R(1) - f;
        R f2 = f * f, f3 = f2 * f;
        w[0] = g * g * g * R(1.0 / 6.0);
        w[1] = (R(3) * f3 - R(6) * f2 + R(4)) * R(1.0 / 6.0);
        w[2] = (R(-3) * f3 + R(3) * f2 + R(3) * f + R(1)) * R(1.0 / 6.0);
        w[3] = f3 * R(1.0 / 6.0);
    }
}

// Support start and weights for a position xi (cell units, in some integer
// frame) on integer nodes (half = false) or on half-integer nodes i+1/2
// stored at index i (half = true).
template <int O, typename R>
__device__ __forceinline__ int support(R xi, bool half, R (&w)[O + 1]) {
    R y = xi - (half ? R(0.5 * O) : R(0.5 * (O - 1)));
    R fl = floor(y);
    bspline<O, R>(y - fl, w);
    return (int)fl;
}

// ---------------------------------------------------------------------------
// Relativistic pushers (Sec. III "Particle motion"), c = 1.
// qmdt = q dt / m.  u: proper velocity at t - dt/2 in, t + dt/2 out.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void push_vay(R qmdt, const R (&E)[3], const R (&B)[3], R (&u)[3]) {
    R ginv = R(1) / sqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    R h = R(0.5) * qmdt;
    R tx = h * B[0], ty = h * B[1], tz = h * B[2];
    // u' = u + qdt/m E + v x tau
    R vx = u[0] * ginv, vy = u[1] * ginv, vz = u[2] * ginv;
    R px = u[0] + qmdt * E[0] + (vy * tz - vz * ty);
    R py = u[1] + qmdt * E[1] + (vz * tx - vx * tz);
    R pz = u[2] + qmdt * E[2] + (vx * ty - vy * tx);
    R tau2 = tx * tx + ty * ty + tz * tz;
    R us = px * tx + py * ty + pz * tz;
    R sigma = R(1) + px * px + py * py + pz * pz - tau2;
    R gnew = sqrt(R(0.5) * (sigma + sqrt(sigma * sigma + R(4) * (tau2 + us * us))));
    R gi = R(1) / gnew;
    tx *= gi; ty *= gi; tz *= gi;
    R s = R(1) / (R(1) + tx * tx + ty * ty + tz * tz);
    R pt = px * tx + py * ty + pz * tz;
    u[0] = s * (px + pt * tx + (py * tz - pz * ty));
    u[1] = s * (py + pt * ty + (pz * tx - px * tz));
    u[2] = s * (pz + pt * tz + (px * ty - py * tx));
}

template <typename R>
__device__ __forceinline__ void push_boris(R qmdt, const R (&E)[3], const R (&B)[3], R (&u)[3]) {
    R h = R(0.5) * qmdt;
    R mx = u[0] + h * E[0], my = u[1] + h * E[1], mz = u[2] + h * E[2];
    R gi = R(1) / sqrt(R(1) + mx * mx + my * my + mz * mz);
    R tx = h * B[0] * gi, ty = h * B[1] * gi, tz = h * B[2] * gi;
    R ax = mx + (my * tz - mz * ty);
    R ay = my + (mz * tx - mx * tz);
    R az = mz + (mx * ty - my * tx);
    R f = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
    R sx = f * tx, sy = f * ty, sz = f * tz;
    u[0] = mx + (ay * sz - az * sy) + h * E[0];
    u[1] = my + (az * sx - ax * sz) + h * E[1];
    u[2] = mz + (ax * sy - ay * sx) + h * E[2];
}

// ---------------------------------------------------------------------------
// Radiative cooling (Sec. "Radiative cooling", eq:prad, eq:udot), explicit and
// not iterated: with p- = um (t - dt/2) and p+^EM = u from the Lorentz push,
// p0 = (p+^EM + p-)/2, gamma0 = sqrt(1 + p0^2) and D = p+^EM - p- = pdot0 dt,
//   p+ = p+^EM - (K/dt) gamma0 (D^2 + |D x p0|^2) / p0^2 * p0,
// K = mu0 q^2 / (6 pi m c) (c = 1); kdt = K / dt.  p0 = 0 does not radiate.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void radiate(R kdt, const R (&um)[3], R (&u)[3]) {
    R px = R(0.5) * (u[0] + um[0]), py = R(0.5) * (u[1] + um[1]), pz = R(0.5) * (u[2] + um[2]);
    R dx = u[0] - um[0], dy = u[1] - um[1], dz = u[2] - um[2];
    R p2 = px * px + py * py + pz * pz;
    if (p2 > R(0)) {
        R cx = dy * pz - dz * py, cy = dz * px - dx * pz, cz = dx * py - dy * px;
        R bracket = dx * dx + dy * dy + dz * dz + (cx * cx + cy * cy + cz * cz);
        R f = -kdt * sqrt(R(1) + p2) * bracket / p2;
        u[0] += f * px;
        u[1] += f * py;
        u[2] += f * pz;
    }
}

// The particle's momentum update: Vay or Boris push, then radiative cooling
// when the species radiates (kdt != 0, uniform over a launch).
template <int PUSH, typename R>
__device__ __forceinline__ void push_particle(R qmdt, R kdt, const R (&E)[3], const R (&B)[3], R (&u)[3]) {
    if (kdt != R(0)) {
        R um[3] = {u[0], u[1], u[2]};
        if (PUSH == PP_BORIS) push_boris<R>(qmdt, E, B, u);
        else push_vay<R>(qmdt, E, B, u);
        radiate<R>(kdt, um, u);
    } else {
        if (PUSH == PP_BORIS) push_boris<R>(qmdt, E, B, u);
        else push_vay<R>(qmdt, E, B, u);
    }
}

// ---------------------------------------------------------------------------
// Gather of one staggered component (eq:pfields): separable triple sum over
// the (O+1)^3 support, x innermost.  Acc::F(kind, comp, i, j, k) reads the
// field at frame indices; kind 0 = E, 1 = B.
// ---------------------------------------------------------------------------
template <int O, typename R, class Acc>
__device__ __forceinline__ R gather_one(const Acc &acc, int kind, int comp, int i0, int j0, int k0,
                                        const R (&wx)[O + 1], const R (&wy)[O + 1], const R (&wz)[O + 1]) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k <= O; ++k) {
        R sy = R(0);
#pragma unroll
        for (int j = 0; j <= O; ++j) {
            R sx = R(0);
#pragma unroll
            for (int i = 0; i <= O; ++i) sx += wx[i] * acc.F(kind, comp, i0 + i, j0 + j, k0 + k);
            sy += wy[j] * sx;
        }
        s += wz[k] * sy;
    }
    return s;
}

template <int O, typename R, class Acc>
__device__ __forceinline__ void gather_EB(const Acc &acc, const R (&xi)[3], R (&E)[3], R (&B)[3]) {
    R wI[3][O + 1], wH[3][O + 1];
    int iI[3], iH[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        iI[a] = support<O, R>(xi[a], false, wI[a]);
        iH[a] = support<O, R>(xi[a], true, wH[a]);
    }
    // E_a: half-integer along a; B_a: integer along a, half-integer across.
    E[0] = gather_one<O, R>(acc, 0, 0, iH[0], iI[1], iI[2], wH[0], wI[1], wI[2]);
    E[1] = gather_one<O, R>(acc, 0, 1, iI[0], iH[1], iI[2], wI[0], wH[1], wI[2]);
    E[2] = gather_one<O, R>(acc, 0, 2, iI[0], iI[1], iH[2], wI[0], wI[1], wH[2]);
    B[0] = gather_one<O, R>(acc, 1, 0, iI[0], iH[1], iH[2], wI[0], wH[1], wH[2]);
    B[1] = gather_one<O, R>(acc, 1, 1, iH[0], iI[1], iH[2], wH[0], wI[1], wH[2]);
    B[2] = gather_one<O, R>(acc, 1, 2, iH[0], iH[1], iI[2], wH[0], wH[1], wI[2]);
}

// ---------------------------------------------------------------------------
// Charge-conserving deposit of one particle (Sec. III, eq:cc1 / eq:jj3 with
// Esirkepov's decomposition) written directly as the 2nd-order current:
// J_a(face lo_a+m+1/2, lo_b+mb, lo_c+mc) = jscale_a * C_a[m] * Y_a[mb][mc],
// C_a[m] = sum_{m' <= m} dS_a[m'] (the per-particle prefix sum along a),
// Y_a = S0_b S0_c + dS_b S0_c / 2 + S0_b dS_c / 2 + dS_b dS_c / 3,
// jscale_a = -q w dx_a / dt.  xi0/xi1: old/new position in the frame of Acc.
// Acc::addJ(comp, i, j, k, v) accumulates into the current of the frame.
// ---------------------------------------------------------------------------
// Weights of one particle's move on the union support of its old and new
// positions: S0 (old) and DS (new - old), O+2 points per axis from lo.
template <int O, typename R>
__device__ __forceinline__ void esirkepov_weights(const R (&xi0)[3], const R (&xi1)[3], R (&S0)[3][O + 2],
                                                  R (&DS)[3][O + 2], int (&lo)[3]) {
    constexpr int S = O + 2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R wo[O + 1], wn[O + 1];
        int io = support<O, R>(xi0[a], false, wo);
        int in = support<O, R>(xi1[a], false, wn);
        int l = io < in ? io : in;
        bool so = io != l, sn = in != l;
#pragma unroll
        for (int m = 0; m < S; ++m) {
            R a0 = so ? (m >= 1 ? wo[m - 1] : R(0)) : (m <= O ? wo[m] : R(0));
            R a1 = sn ? (m >= 1 ? wn[m - 1] : R(0)) : (m <= O ? wn[m] : R(0));
            S0[a][m] = a0;
            DS[a][m] = a1 - a0;
        }
        lo[a] = l;
    }
}

// Fixed-point current windows (the tiled kernels): largest |C[m] Y[mb][mc]| of
// one particle per unit of its displacement |dxi_a|.  C[m] is a difference of
// two values of the cumulative sum of W^O over the nodes up to the face, a
// function of position whose slope is a W^(O-1) value, so |C| <= |dxi_a|
// max W^(O-1); Y = S0b S0c/3 + S1b S0c/6 + S0b S1c/6 + S1b S1c/3 is a convex
// combination of products of weights, so 0 <= Y <= (max W^O)^2.  With
// max W^0 = max W^1 = 1, max W^2 = 3/4 and max W^3 = 2/3 (Sec. II list after
// eq:weightfunction) the product is 1, 9/16 and 1/3 for O = 1, 2, 3.  The
// direct current's q w v W W W per unit displacement is at most (max W^O)^3,
// below the same figure.
template <int O>
__host__ __device__ constexpr float fixed_point_cy_bound() {
    return O == 1 ? 1.0f : (O == 2 ? 0.5625f : 1.0f / 3.0f);
}

// Component A of the current of one particle from its weights.
template <int O, typename R, int A, class Acc>
__device__ __forceinline__ void esirkepov_component(Acc &acc, const R (&S0)[3][O + 2], const R (&DS)[3][O + 2],
                                                    const int (&lo)[3], R jscale) {
    constexpr int S = O + 2;
    constexpr int B = (A + 1) % 3, Cc = (A + 2) % 3;
    // C[m] = sum_{m' <= m} dS[m'] = -sum_{m' > m} dS[m'] (the support sums
    // to zero): the upper faces use the suffix form, so a particle that
    // stays inside its cell gets exact zeros there.
    R C[O + 1];
    R run = R(0);
#pragma unroll
    for (int m = 0; m <= O; ++m) {
        if (2 * m < O + 1) {
            run += DS[A][m];
            C[m] = run * jscale;
        }
    }
    run = R(0);
#pragma unroll
    for (int m = O; m >= 0; --m) {
        if (2 * m >= O + 1) {
            run -= DS[A][m + 1];
            C[m] = run * jscale;
        }
    }
#pragma unroll
    for (int mc = 0; mc < S; ++mc) {
        R p = S0[Cc][mc] + R(0.5) * DS[Cc][mc];
        R q = R(0.5) * S0[Cc][mc] + R(1.0 / 3.0) * DS[Cc][mc];
#pragma unroll
        for (int mb = 0; mb < S; ++mb) {
            R Y = S0[B][mb] * p + DS[B][mb] * q;
#pragma unroll
            for (int m = 0; m <= O; ++m) {
                R v = C[m] * Y;
                if (v == R(0)) continue;
                int idx[3];
                idx[A] = lo[A] + m;
                idx[B] = lo[B] + mb;
                idx[Cc] = lo[Cc] + mc;
                acc.addJ(A, idx[0], idx[1], idx[2], v);
            }
        }
    }
}

template <int O, typename R, class Acc>
__device__ __forceinline__ void deposit_esirkepov(Acc &acc, const R (&xi0)[3], const R (&xi1)[3],
                                                  const R (&jscale)[3]) {
    R S0[3][O + 2], DS[3][O + 2];
    int lo[3];
    esirkepov_weights<O, R>(xi0, xi1, S0, DS, lo);
    esirkepov_component<O, R, 0>(acc, S0, DS, lo, jscale[0]);
    esirkepov_component<O, R, 1>(acc, S0, DS, lo, jscale[1]);
    esirkepov_component<O, R, 2>(acc, S0, DS, lo, jscale[2]);
}

// deposit_esirkepov for a particle whose old and new positions share the
// support start on every axis (it crosses no support boundary in the step):
// the union support is the O+1 points of both, the prefix C vanishes on the
// last face, and each component has O (O+1)^2 sites.  The products are those
// of deposit_esirkepov site by site (its zero sites are left out here, its
// skipped exact zeros are added here).  Returns false, depositing nothing,
// for any other particle.
template <int O, typename R, class Acc>
__device__ __forceinline__ bool deposit_esirkepov_inner(Acc &acc, const R (&xi0)[3], const R (&xi1)[3],
                                                        const R (&jscale)[3]) {
    R S0[3][O + 1], DS[3][O + 1];
    int lo[3];
    bool same = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R wo[O + 1], wn[O + 1];
        int io = support<O, R>(xi0[a], false, wo);
        int in = support<O, R>(xi1[a], false, wn);
        same = same && io == in;
        lo[a] = io;
#pragma unroll
        for (int m = 0; m <= O; ++m) {
            S0[a][m] = wo[m];
            DS[a][m] = wn[m] - wo[m];
        }
    }
    if (!same) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        R C[O];
        R run = R(0);
#pragma unroll
        for (int m = 0; m < O; ++m) {
            if (2 * m < O + 1) {
                run += DS[a][m];
                C[m] = run * jscale[a];
            }
        }
        run = R(0);   // C[O] = -DS[O+1] = 0: the suffix starts below it
#pragma unroll
        for (int m = O - 1; m >= 0; --m) {
            if (2 * m >= O + 1) {
                run -= DS[a][m + 1];
                C[m] = run * jscale[a];
            }
        }
#pragma unroll
        for (int mc = 0; mc <= O; ++mc) {
            R p = S0[c][mc] + R(0.5) * DS[c][mc];
            R q = R(0.5) * S0[c][mc] + R(1.0 / 3.0) * DS[c][mc];
#pragma unroll
            for (int mb = 0; mb <= O; ++mb) {
                R Y = S0[b][mb] * p + DS[b][mb] * q;
#pragma unroll
                for (int m = 0; m < O; ++m) {
                    int idx[3];
                    idx[a] = lo[a] + m;
                    idx[b] = lo[b] + mb;
                    idx[c] = lo[c] + mc;
                    acc.addJ(a, idx[0], idx[1], idx[2], C[m] * Y);
                }
            }
        }
    }
    return true;
}

// Direct current of one particle (eq:jj2, the paper's original method):
// q w v W(x_mid - x_c) on each component's staggered nodes (staggered like E),
// with x_mid = xi0 + dxi / 2 in the frame of Acc and q w v_a = -jscale_a dxi_a
// (jscale_a = -q w dx_a / dt).  No continuity: see eq:cc1 for why the paper
// replaced it.
template <int O, typename R, class Acc>
__device__ __forceinline__ void deposit_direct(Acc &acc, const R (&xi0)[3], const R (&dxi)[3], const R (&jscale)[3]) {
    R wI[3][O + 1], wH[3][O + 1];
    int iI[3], iH[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R xm = xi0[a] + R(0.5) * dxi[a];
        iI[a] = support<O, R>(xm, false, wI[a]);
        iH[a] = support<O, R>(xm, true, wH[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R vs = -jscale[a] * dxi[a];
        const R *wx = a == 0 ? wH[0] : wI[0], *wy = a == 1 ? wH[1] : wI[1], *wz = a == 2 ? wH[2] : wI[2];
        const int i0 = a == 0 ? iH[0] : iI[0], j0 = a == 1 ? iH[1] : iI[1], k0 = a == 2 ? iH[2] : iI[2];
#pragma unroll
        for (int k = 0; k <= O; ++k) {
            R vz = vs * wz[k];
#pragma unroll
            for (int j = 0; j <= O; ++j) {
                R vyz = vz * wy[j];
#pragma unroll
                for (int i = 0; i <= O; ++i) acc.addJ(a, i0 + i, j0 + j, k0 + k, vyz * wx[i]);
            }
        }
    }
}

// Charge weights of one particle on the integer nodes (eq:rho2).
template <int O, typename R, class Acc>
__device__ __forceinline__ void deposit_rho(Acc &acc, const R (&xi)[3], R qw) {
    R w[3][O + 1];
    int i0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) i0[a] = support<O, R>(xi[a], false, w[a]);
#pragma unroll
    for (int k = 0; k <= O; ++k)
#pragma unroll
        for (int j = 0; j <= O; ++j)
#pragma unroll
            for (int i = 0; i <= O; ++i) acc.addRho(i0[0] + i, i0[1] + j, i0[2] + k, qw * w[0][i] * w[1][j] * w[2][k]);
}

// ---------------------------------------------------------------------------
// Context (host side)
// ---------------------------------------------------------------------------
struct Species {
    double q, m, w;
    double rad = 0.0;         // radiative-cooling coefficient mu0 q^2 / (6 pi m c); 0 = off
    int64_t cap = 0, n = 0;   // allocated slots (rounded up to 64) and particles held
    int64_t limit = 0;        // capacity requested by the caller
    // PP_FP64: positions in cell units xi = x/dx in [0, n); momenta
    double *x = nullptr, *y = nullptr, *z = nullptr, *ux = nullptr, *uy = nullptr, *uz = nullptr;
    // PP_MIXED32: packed cell (x | y << 10 | z << 20) + FP32 offsets and momenta
    int32_t *cell = nullptr;
    float *ox = nullptr, *oy = nullptr, *oz = nullptr, *fux = nullptr, *fuy = nullptr, *fuz = nullptr;
    int64_t nsorted = 0;      // particles [0, nsorted) are in cell_start's ranges; the rest
                              // (injected since the last sort) form an unsorted tail
    bool may_hold_dead = false;   // particles may have left (escape, window) since the last sort
    void *buf = nullptr;      // primary particle storage
    void *alt = nullptr;      // sort target of the same layout
    int32_t *keys = nullptr;  // sort keys
    int32_t *cell_start = nullptr; // offsets per sort key (nkeys + 1), valid after a sort
    bool sorted = false;
    bool fresh = false;       // sorted since the particles last moved (the per-step sorted kernel needs it)
    // Per-step sorted kernel: its pass writes every particle's new sort key
    // (keys_valid), and the sort that follows only builds the permutation
    // perm (perm_pending: slot i of the sorted order holds particle perm[i]),
    // which the next pass applies while it reads the particles.  Any other
    // reader of the particle arrays first applies it (materialize).
    int32_t *perm = nullptr;
    bool perm_pending = false;
    bool keys_valid = false;
    // Point the SoA arrays into buf (the sort swaps buf and alt).
    void bind(bool fp64) {
        if (fp64) {
            double *b = (double *)buf;
            x = b; y = b + cap; z = b + 2 * cap; ux = b + 3 * cap; uy = b + 4 * cap; uz = b + 5 * cap;
        } else {
            int32_t *ci = (int32_t *)buf;
            float *f = (float *)(ci + cap);
            cell = ci; ox = f; oy = f + cap; oz = f + 2 * cap; fux = f + 3 * cap; fuy = f + 4 * cap; fuz = f + 5 * cap;
        }
    }
};

// One step captured as a CUDA graph (pp_set_graphs).  A step's launches and
// their pointer arguments are fixed by the state it starts from: whether it
// sorts, which of J / J' holds the current, and which buffer holds each
// species (the sort swaps them).  The host-side state the step leaves behind
// is stored with it and re-applied on every replay.
struct StepGraph {
    bool valid = false;
    bool sort = false;
    void *J0 = nullptr;
    void *buf[PP_MAX_SPECIES] = {};
    bool sorted[PP_MAX_SPECIES] = {};
    bool fresh[PP_MAX_SPECIES] = {};
    bool pending[PP_MAX_SPECIES] = {}, keys_valid[PP_MAX_SPECIES] = {};
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    bool filter = false;
    void *J_after[3] = {}, *Jt_after[3] = {};
    void *buf_after[PP_MAX_SPECIES] = {}, *alt_after[PP_MAX_SPECIES] = {};
    bool sorted_after[PP_MAX_SPECIES] = {}, fresh_after[PP_MAX_SPECIES] = {};
    bool pending_after[PP_MAX_SPECIES] = {}, keys_valid_after[PP_MAX_SPECIES] = {};
    int since_sort_after = 0;
    int last_iters = 0;
    double last_kk = 0;
    bool filtered_after_solve = false;
};
constexpr int kGraphSlots = 8;

enum Phase { PH_PARTICLE = 0, PH_CURRENT = 1, PH_FIELD = 2, PH_SORT = 3, PH_N = 4 };

struct EventPair {
    int phase;
    cudaEvent_t a, b;
};

struct Ctx {
    pp_grid_desc d;
    cudaStream_t st = nullptr;
    Geom g;
    bool fp64 = true;
    size_t rsz = 8;
    void *mesh = nullptr;
    void *E[3], *B[3], *J[3], *Jt[3], *R[3], *Xa[3], *Xb[3];
    double *rho = nullptr;   // compact FP64 charge density (diagnostics)
    double *G0 = nullptr;    // compact FP64 Gauss reference
    bool have_G0 = false;
    // high-order current: symmetric circulant taps of the inverse of the
    // (c, b+c, a+b+c, b+c, c) line operator, per axis
    double *taps = nullptr;  // device, 3 x kMaxTaps
    int ntaps[3] = {0, 0, 0};
    bool full_circ[3] = {false, false, false};
    // field solve
    double fd[3];            // a, b, c
    double lap[6];           // 1D stencil of d^+ d^- at offsets 0..5
    struct Cheb {            // Chebyshev semi-iteration on the spectrum [1, 2 theta - 1]
        double theta = 1, delta = 0;
        int iters = 0;
    };
    Cheb cheb[3];            // solve step |dt|, |a_1| dt, |a_2| dt (4th-order substeps)
    int cheb_sel = 0;        // the set the next field update uses
    int last_iters = 0;
    double last_kk = 0;      // alpha^2 dt^2 of the last solve
    // time integration: order 2 = leap-frog step; 4 = four kick-drift substeps
    // (Sec. III, symmetric fourth-order integrator).  kick_dt / drift_dt are
    // the sizes of the (sub)step being taken; both equal dt outside a
    // 4th-order step.
    int order = 2;
    double kick_dt = 0, drift_dt = 0;
    int field_solver = 0;    // PP_FIELD_IMPLICIT or PP_FIELD_EXPLICIT
    bool g0_pending = false; // a load changed rho or E: take the Gauss reference before the next use
    int current_mode = 0;    // PP_CURRENT_CONSERVING or PP_CURRENT_DIRECT
    // Reflecting walls at 0 and wall[a] (cells) on axis a: the mesh is the
    // mirror-extended box there, g.n[a] = 2 * wall[a].  0 = periodic.  The open
    // end, the injectors and the window act on x and need wall[0].
    int wall[3] = {0, 0, 0};
    bool any_wall() const { return wall[0] || wall[1] || wall[2]; }
    // Open lower end between walls (outflow layer, escape), injectors and the
    // sliding window (Sec. V "Boundary conditions", "Sliding window and
    // injection of particles").
    struct OpenEnd {
        int cells = 0;           // damping layer width; 0 = no open end
        double damping = 0.0;    // factor 1 - damping ((cells - d) / cells)^2 per step
        double escape = 0.0;     // outgoing particles closer than this (cells) leave
        int mask = 0;            // damped components: bit a = E_a, bit 3 + a = B_a
    } open;
    struct Injector {
        double ppc = 0.0;        // particles per cell of the inflow; 0 = off
        double u[3] = {0, 0, 0}; // drift proper velocity
        double u_th = 0.0;
        uint64_t seed = 0;
        int64_t k0 = 0;          // step at which it was set
    } inj[PP_MAX_SPECIES];
    struct Window {
        double v = 0.0;          // speed against x; 0 = off
        int64_t k0 = 0;
        int64_t shifts = 0;
    } window;
    int32_t *h_count = nullptr;  // pinned: live count read back after a compacting sort
    // z-slab decomposition: this context owns the particles with physical z in
    // [slab_lo, slab_hi) of a run split over ranks (pp_set_slab)
    bool slab = false;
    double slab_lo = 0.0, slab_hi = 0.0;
    double escape_now = 0.0;     // escape distance the particle kernels apply (0: none this pass)
    int filter_passes = 0;   // divergence-filter passes every filter_interval steps
    int filter_interval = 1;
    double filter_tau = 0;   // 1 / largest eigenvalue of -div grad
    bool filtered_after_solve = false;   // a filter changed B after the last relaxation
    // step graphs
    bool use_graphs = false;
    StepGraph graphs[kGraphSlots];
    int graph_next = 0;          // slot replaced on the next miss when all are valid
    int64_t graph_captures = 0, graph_replays = 0;
    // sort
    int tile[3] = {8, 8, 8};
    int ntile[3] = {1, 1, 1};
    int64_t nkeys = 0;
    int32_t *counts = nullptr;   // nkeys + 1
    void *scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    int since_sort = 0;
    // status
    int *d_status = nullptr;
    int *h_status = nullptr;     // pinned mirror
    unsigned long long *d_nslow = nullptr;
    unsigned *d_slow_count = nullptr;   // per species, particles left to the global-mesh kernel
    // reductions
    double *d_red = nullptr;     // partials
    double *d_out = nullptr;     // final values
    int64_t step = 0;
    // profiling (pp_profile_enable / pp_profile_read)
    bool prof = false;
    EventPair *prof_ev = nullptr;
    int prof_n = 0, prof_cap = 0;
    double prof_ms[PH_N] = {0, 0, 0, 0};
    int64_t prof_particle_launches = 0, prof_steps = 0;
    int64_t nlaunch = 0;          // kernels enqueued (counted by the launchers)
    int nspecies = 0;
    Species sp[PP_MAX_SPECIES];
    char err[512] = {0};
};

constexpr int kMaxTaps = 64;

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files); all enqueue on c.st.
// ---------------------------------------------------------------------------
cudaError_t launch_particles_fp64(Ctx &c, int s);
cudaError_t launch_particles_mixed_global(Ctx &c, int s);
cudaError_t launch_particles_tiled_all(Ctx &c);
bool tiled_supported(const Ctx &c);
cudaError_t launch_particles_cells(Ctx &c);
bool cells_supported(const Ctx &c);
// batched form: one launch over the tiles of many contexts (same shape order,
// pusher and boundary kind); scratch = device memory the caller owns
struct CellsBatchScratch {
    void *args = nullptr;   // per context argument block
    void *items = nullptr;  // (context, tile) work items
    int *next = nullptr;    // work counter
    size_t args_cap = 0, items_cap = 0;
};
int cells_batch_key(const Ctx &c);   // contexts with equal keys can share a launch
cudaError_t launch_particles_cells_batch(Ctx *const *ctxs, int n, cudaStream_t st, CellsBatchScratch &scr,
                                         void *host_args, void *host_items, int nsm);
size_t cells_args_bytes();
bool batch_fusable(const Ctx *c);
int batch_step_pre(Ctx *c);
int batch_step_post(Ctx *c);
// sort_first (calls outside a step: diagnostics, the Gauss reference, rho
// readback): a mixed-form species whose particles are unsorted, or that the
// per-step sorted kernel left with fresh keys, is sorted first, so that every
// particle sits in its sorted cell and the tile kernel adds none directly.
cudaError_t launch_rho(Ctx &c, bool sort_first = false);
cudaError_t launch_kinetic(Ctx &c, double *out_per_species);

cudaError_t launch_zero_J(Ctx &c);
cudaError_t launch_fold_J(Ctx &c);
cudaError_t launch_mirror_J(Ctx &c);
cudaError_t launch_mirror_fields(Ctx &c);
cudaError_t launch_mirror_rho(Ctx &c, double *rho);
cudaError_t launch_current_solve(Ctx &c);
cudaError_t launch_field_update(Ctx &c);
cudaError_t launch_divergence_filter(Ctx &c);
cudaError_t launch_ghost_fill(Ctx &c, void *const src_E[3], void *const src_B[3]);
cudaError_t launch_mesh_diag(Ctx &c, double *host_out /* 9 values */);

cudaError_t launch_sort(Ctx &c, int s);
cudaError_t materialize(Ctx &c, int s);   // apply a pending sort permutation to the arrays
cudaError_t launch_damp(Ctx &c);
cudaError_t launch_inject(Ctx &c, int s, int64_t off, int64_t count, uint32_t step, uint32_t pstream, double thick);
cudaError_t launch_window_fields(Ctx &c);
cudaError_t launch_window_particles(Ctx &c, int s);
cudaError_t sort_setup(Ctx &c);

cudaError_t launch_convert_in(Ctx &c, int s, int64_t off, int64_t n, const double *x, const double *y,
                              const double *z, const double *ux, const double *uy, const double *uz, int *bad);
cudaError_t launch_convert_out(Ctx &c, int s, double *x, double *y, double *z, double *ux, double *uy,
                               double *uz);
cudaError_t launch_extract(Ctx &c, int s, double z_lo, double z_hi, int write, int64_t cap,
                           unsigned long long *count, double *const out[6]);

}  // namespace pp
