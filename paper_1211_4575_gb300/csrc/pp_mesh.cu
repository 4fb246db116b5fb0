// pp_mesh.cu -- mesh kernels of the step: periodic ghost fold of the deposited
// current, the high-order current solve (Sec. III eq:jj6 .. eq:penta), the
// implicit de-centred field update (eq:bnplus1, eq:enplus1, eq:EllipticB),
// the periodic ghost fill of E and B, and the FP64 mesh diagnostics.
//
// Mesh arrays are padded (Geom::at).  E and B keep their periodic ghost layers
// filled (the particle gather reads them), and so do the relaxation iterates:
// the implicit solver's stencils read those through linear offsets (NbLin).
// Other stencils read interior values through periodic wrapping (Nb).
#include "pp_internal.cuh"

namespace pp {

__device__ __forceinline__ void unflatten(int64_t t, const Geom &g, int &i, int &j, int &k) {
    i = (int)(t % g.n[0]);
    int64_t r = t / g.n[0];
    j = (int)(r % g.n[1]);
    k = (int)(r / g.n[1]);
}

// ---------------------------------------------------------------------------
// Ghost fold: every interior node collects the ghost images of itself along
// one axis (coordinate + m*n, m != 0, inside the padding) and the ghosts are
// cleared.  Passes x, y, z in turn; each ghost is read by exactly one thread.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_fold_axis(Geom g, R *J0, R *J1, R *J2, int axis, int lo0, int lo1, int lo2, int e0, int e1,
                            int e2) {
    int64_t total = (int64_t)e0 * e1 * e2;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int c[3];
    c[0] = lo0 + (int)(t % e0);
    int64_t r = t / e0;
    c[1] = lo1 + (int)(r % e1);
    c[2] = lo2 + (int)(r / e1);
    R *Js[3] = {J0, J1, J2};
    int n = g.n[axis];
    int64_t base = g.at(c[0], c[1], c[2]);
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)g.P[0] : (int64_t)g.P[0] * g.P[1]);
    int x = c[axis];
    for (int comp = 0; comp < 3; ++comp) {
        R *J = Js[comp];
        R acc = J[base];
        for (int m = -((g.G + n - 1) / n); m <= (g.G + n - 1) / n; ++m) {
            if (m == 0) continue;
            int y = x + m * n;
            if (y < -g.G || y >= n + g.G) continue;
            int64_t q = base + (int64_t)(y - x) * stride;
            acc += J[q];
            J[q] = R(0);
        }
        J[base] = acc;
    }
}

template <typename R>
static cudaError_t fold_impl(Ctx &c) {
    const Geom &g = c.g;
    int G = g.G;
    R *J0 = (R *)c.J[0], *J1 = (R *)c.J[1], *J2 = (R *)c.J[2];
    // x pass over padded y, z; y pass over interior x, padded z; z pass over interior x, y
    int lo[3][3] = {{0, -G, -G}, {0, 0, -G}, {0, 0, 0}};
    int ex[3][3] = {{g.n[0], g.n[1] + 2 * G, g.n[2] + 2 * G}, {g.n[0], g.n[1], g.n[2] + 2 * G}, {g.n[0], g.n[1], g.n[2]}};
    for (int a = 0; a < 3; ++a) {
        int64_t total = (int64_t)ex[a][0] * ex[a][1] * ex[a][2];
        k_fold_axis<R><<<(unsigned)((total + 255) / 256), 256, 0, c.st>>>(g, J0, J1, J2, a, lo[a][0], lo[a][1], lo[a][2],
                                                                          ex[a][0], ex[a][1], ex[a][2]);
        ++c.nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fold_J(Ctx &c) { return c.fp64 ? fold_impl<double>(c) : fold_impl<float>(c); }

cudaError_t launch_zero_J(Ctx &c) {
    size_t bytes = (size_t)c.g.padded_size() * c.rsz;
    for (int a = 0; a < 3; ++a) {
        cudaError_t e = cudaMemsetAsync(c.J[a], 0, bytes, c.st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Reflecting walls (Sec. V "Boundary conditions").  On a walled axis a the
// mesh is the mirror-extended box of n0 = 2 n_a cells, the walls on the
// integer nodes 0 and n_a.  Along a, integer node i has the image
// (n0 - i) mod n0 and half node i+1/2 (index i) the image index n0 - 1 - i.
// Components staggered along a are odd across the wall and the others even:
// E_a and J_a, and every B_b with b != a.  Walls on several axes fold one axis
// after the other (the images of images are the corner images).
//
// avg = 0 (a deposit): the virtual images contribute the mirror of what the
// particles deposited, f(i) <- f(i) + P f(m(i)), and the image node receives
// P times that sum; a wall node, its own image, doubles.  avg = 1 (a load):
// f(i) <- (f(i) + P f(m(i))) / 2 on both nodes of the pair.  One thread per
// pair: i in [0, n_a] along a row (odd components stop at n_a - 1).
// ---------------------------------------------------------------------------
struct PaddedIndex {
    Geom g;
    __device__ __forceinline__ int64_t operator()(int i, int j, int k) const { return g.at(i, j, k); }
};
struct CompactIndex {
    int n0, n1;
    __device__ __forceinline__ int64_t operator()(int i, int j, int k) const {
        return i + (int64_t)n0 * (j + (int64_t)n1 * k);
    }
};

// Pairs along the wall normal `ax` (walls at 0 and nw cells), over the mesh
// extents ne of the other two axes: thread (i, p, r) holds the row position i
// along ax and the coordinates p, r along axes ax+1, ax+2 (mod 3).
template <typename R, class Ix>
__global__ void k_mirror(Ix ix, int ax, int nw, int nb, int nc, R *F0, R *F1, R *F2, int odd_mask, int avg) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int comp = blockIdx.y;
    if (t >= (int64_t)(nw + 1) * nb * nc) return;
    const int i = (int)(t % (nw + 1));
    const int64_t r = t / (nw + 1);
    const int pb = (int)(r % nb), pc = (int)(r / nb);
    const bool odd = (odd_mask >> comp) & 1;
    int m;
    if (odd) {
        if (i == nw) return;
        m = 2 * nw - 1 - i;
    } else {
        m = i == 0 ? 0 : 2 * nw - i;
    }
    int q[3], qm[3];
    q[ax] = i;
    qm[ax] = m;
    q[(ax + 1) % 3] = qm[(ax + 1) % 3] = pb;
    q[(ax + 2) % 3] = qm[(ax + 2) % 3] = pc;
    R *F = comp == 0 ? F0 : (comp == 1 ? F1 : F2);
    const int64_t a = ix(q[0], q[1], q[2]), b = ix(qm[0], qm[1], qm[2]);
    const R P = odd ? R(-1) : R(1);
    R v = F[a] + P * F[b];
    if (avg) v *= R(0.5);
    F[a] = v;
    if (b != a) F[b] = P * v;
}

// Components odd across a wall with normal ax: E_ax and J_ax (staggered along
// it); for B every component but B_ax.
static inline int odd_mask(bool bfield, int ax) { return bfield ? (7 & ~(1 << ax)) : (1 << ax); }

template <typename R, class Ix>
static cudaError_t mirror_axes(Ctx &c, Ix ix, R *F0, R *F1, R *F2, int ncomp, int bfield_or_rho, int avg) {
    for (int ax = 0; ax < 3; ++ax) {
        const int nw = c.wall[ax];
        if (!nw) continue;
        const int nb = c.g.n[(ax + 1) % 3], nc = c.g.n[(ax + 2) % 3];
        const int mask = bfield_or_rho < 0 ? 0 : odd_mask(bfield_or_rho == 1, ax);
        dim3 grid((unsigned)(((int64_t)(nw + 1) * nb * nc + 255) / 256), (unsigned)ncomp);
        k_mirror<R, Ix><<<grid, 256, 0, c.st>>>(ix, ax, nw, nb, nc, F0, F1, F2, mask, avg);
        ++c.nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R>
static cudaError_t mirror_padded(Ctx &c, void *const F[3], int bfield, int avg) {
    return mirror_axes<R, PaddedIndex>(c, PaddedIndex{c.g}, (R *)F[0], (R *)F[1], (R *)F[2], 3, bfield, avg);
}

cudaError_t launch_mirror_J(Ctx &c) {
    if (!c.any_wall()) return cudaSuccess;
    return c.fp64 ? mirror_padded<double>(c, c.J, 0, 0) : mirror_padded<float>(c, c.J, 0, 0);
}

cudaError_t launch_mirror_fields(Ctx &c) {
    if (!c.any_wall()) return cudaSuccess;
    cudaError_t e = c.fp64 ? mirror_padded<double>(c, c.E, 0, 1) : mirror_padded<float>(c, c.E, 0, 1);
    if (e != cudaSuccess) return e;
    return c.fp64 ? mirror_padded<double>(c, c.B, 1, 1) : mirror_padded<float>(c, c.B, 1, 1);
}

cudaError_t launch_mirror_rho(Ctx &c, double *rho) {
    if (!c.any_wall()) return cudaSuccess;
    return mirror_axes<double, CompactIndex>(c, CompactIndex{c.g.n[0], c.g.n[1]}, rho, rho, rho, 1, -1, 0);
}

// ---------------------------------------------------------------------------
// Open lower end (Sec. V "Boundary conditions", outflow): each step the
// chosen components are multiplied by 1 - damping ((cells - d) / cells)^2 at
// distance d < cells from x = 0, d taken at the component's staggered
// position, on both sides of that mirror plane so that the extended mesh stays
// symmetric.  Columns: the first `cells` x-indices and the last `cells`.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_damp(Geom g, R *F, int half, int cells, double damping) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cols = 2 * cells;
    if (t >= (int64_t)cols * g.n[1] * g.n[2]) return;
    const int c = (int)(t % cols);
    const int64_t r = t / cols;
    const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
    const int N = g.n[0];
    const int i = c < cells ? c : N - 2 * cells + c;
    const double pos = i + (half ? 0.5 : 0.0);
    const double d = fmin(pos, N - pos);
    if (d >= cells) return;
    const double s = (cells - d) / cells;
    F[g.at(i, j, k)] *= (R)(1.0 - damping * s * s);
}

template <typename R>
static cudaError_t damp_impl(Ctx &c) {
    const int cells = c.open.cells;
    void **groups[2] = {c.E, c.B};
    const int half[2] = {1, 6};   // staggered in x: E_x; B_y, B_z
    const unsigned blocks = (unsigned)(((int64_t)2 * cells * c.g.n[1] * c.g.n[2] + 255) / 256);
    for (int f = 0; f < 2; ++f)
        for (int comp = 0; comp < 3; ++comp) {
            if (!((c.open.mask >> (3 * f + comp)) & 1)) continue;
            k_damp<R><<<blocks, 256, 0, c.st>>>(c.g, (R *)groups[f][comp], (half[f] >> comp) & 1, cells,
                                                c.open.damping);
            ++c.nlaunch;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    return launch_ghost_fill(c, c.E, c.B);
}

cudaError_t launch_damp(Ctx &c) {
    if (!c.wall[0] || c.open.cells <= 0 || !c.open.mask) return cudaSuccess;
    return c.fp64 ? damp_impl<double>(c) : damp_impl<float>(c);
}

// ---------------------------------------------------------------------------
// Sliding window (Sec. V "Sliding window and injection of particles"): the
// content of the box moves one cell up in x.  In the physical half a node takes
// the value of the node one cell below (zero for the new bottom node); a node
// of the mirror half takes P times the new value of its image.  Written into
// scratch arrays, which then swap with E and B.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_window_fields(Geom g, int nw, const R *I0, const R *I1, const R *I2, R *O0, R *O1, R *O2,
                                int odd_mask) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int comp = blockIdx.y;
    if (t >= g.cells()) return;
    const int i = (int)(t % g.n[0]);
    const int64_t r = t / g.n[0];
    const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
    const bool odd = (odd_mask >> comp) & 1;
    const R *in = comp == 0 ? I0 : (comp == 1 ? I1 : I2);
    R *out = comp == 0 ? O0 : (comp == 1 ? O1 : O2);
    const int top = odd ? nw - 1 : nw;   // last node of the physical half
    int src = i;
    R sign = R(1);
    if (i > top) {                        // mirror half: the image node
        src = odd ? 2 * nw - 1 - i : 2 * nw - i;
        sign = odd ? R(-1) : R(1);
    }
    out[g.at(i, j, k)] = src == 0 ? R(0) : sign * in[g.at(src - 1, j, k)];
}

template <typename R>
static cudaError_t window_fields_impl(Ctx &c) {
    dim3 grid((unsigned)((c.g.cells() + 255) / 256), 3);
    void **F[2] = {c.E, c.B};
    void **S[2] = {c.Xa, c.Xb};
    const int odd[2] = {1, 6};
    for (int f = 0; f < 2; ++f) {
        k_window_fields<R><<<grid, 256, 0, c.st>>>(c.g, c.wall[0], (const R *)F[f][0], (const R *)F[f][1],
                                                   (const R *)F[f][2], (R *)S[f][0], (R *)S[f][1], (R *)S[f][2],
                                                   odd[f]);
        ++c.nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        for (int a = 0; a < 3; ++a) {
            void *t = F[f][a];
            F[f][a] = S[f][a];
            S[f][a] = t;
        }
    }
    return launch_ghost_fill(c, c.E, c.B);
}

cudaError_t launch_window_fields(Ctx &c) {
    if (!c.wall[0]) return cudaSuccess;
    return c.fp64 ? window_fields_impl<double>(c) : window_fields_impl<float>(c);
}

// ---------------------------------------------------------------------------
// High-order current: along the axis of each component, J_out = P^{-1} J_in
// with P the symmetric cyclic line operator (c, b+c, a+b+c, b+c, c) that
// turns the 2nd-order difference into the high-order one; applied as the
// exact (or exponentially truncated) circulant inverse, taps precomputed in
// FP64 on the host.  out(i) = sum_m T[m] * in(i + off + m).
// ---------------------------------------------------------------------------
struct TapSet {
    const double *T[3];
    int L[3];
    int off[3];
};

template <typename R>
__global__ void k_current_solve(Geom g, TapSet ts, const R *I0, const R *I1, const R *I2, R *O0, R *O1, R *O2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int comp = blockIdx.y;
    if (t >= g.cells()) return;
    int c[3];
    unflatten(t, g, c[0], c[1], c[2]);
    const R *in = comp == 0 ? I0 : (comp == 1 ? I1 : I2);
    R *out = comp == 0 ? O0 : (comp == 1 ? O1 : O2);
    const double *T = ts.T[comp];
    int L = ts.L[comp], off = ts.off[comp], n = g.n[comp];
    int x = c[comp];
    R acc = R(0);
    int q[3] = {c[0], c[1], c[2]};
    for (int m = 0; m < L; ++m) {
        q[comp] = wrap(x + off + m, n);
        acc += (R)__ldg(T + m) * in[g.at(q[0], q[1], q[2])];
    }
    out[g.at(c[0], c[1], c[2])] = acc;
}

cudaError_t launch_current_solve(Ctx &c) {
    if (c.d.field_order == 2) return cudaSuccess;
    TapSet ts;
    for (int a = 0; a < 3; ++a) {
        ts.T[a] = c.taps + a * kMaxTaps;
        ts.L[a] = c.ntaps[a];
        ts.off[a] = c.full_circ[a] ? 0 : -(c.ntaps[a] / 2);
    }
    dim3 grid((unsigned)((c.g.cells() + 255) / 256), 3);
    if (c.fp64)
        k_current_solve<double><<<grid, 256, 0, c.st>>>(c.g, ts, (double *)c.J[0], (double *)c.J[1], (double *)c.J[2],
                                                        (double *)c.Jt[0], (double *)c.Jt[1], (double *)c.Jt[2]);
    else
        k_current_solve<float><<<grid, 256, 0, c.st>>>(c.g, ts, (float *)c.J[0], (float *)c.J[1], (float *)c.J[2],
                                                       (float *)c.Jt[0], (float *)c.Jt[1], (float *)c.Jt[2]);
    ++c.nlaunch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a) {
        void *t = c.J[a];
        c.J[a] = c.Jt[a];
        c.Jt[a] = t;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Field update.  Staggered first differences (Sec. III):
//   d^+ f (i+1/2) = sum_m k_m (f[i+m] - f[i+1-m]) / h
//   d^- f (i)     = sum_m k_m (f[i+m-1] - f[i-m]) / h
// and the Laplacian sum_a d^+_a d^-_a as the symmetric 11-point stencil lap[].
// ---------------------------------------------------------------------------
struct FieldCoef {
    double k[3];      // a, b, c
    double lap[6];    // offsets 0..5 of the 1D d^+ d^- stencil (times 1)
    double ih[3];     // 1/h per axis
    double ih2[3];    // 1/h^2 per axis
};

template <typename R>
struct Nb {
    const Geom &g;
    int c[3];
    __device__ __forceinline__ R at(const R *f, int axis, int s) const {
        int q[3] = {c[0], c[1], c[2]};
        q[axis] = wrap(c[axis] + s, g.n[axis]);
        return f[g.at(q[0], q[1], q[2])];
    }
    __device__ __forceinline__ R dplus(const R *f, int axis, const FieldCoef &k) const {
        R s = R(0);
#pragma unroll
        for (int m = 1; m <= 3; ++m) s += (R)k.k[m - 1] * (at(f, axis, m) - at(f, axis, 1 - m));
        return s * (R)k.ih[axis];
    }
    __device__ __forceinline__ R dminus(const R *f, int axis, const FieldCoef &k) const {
        R s = R(0);
#pragma unroll
        for (int m = 1; m <= 3; ++m) s += (R)k.k[m - 1] * (at(f, axis, m - 1) - at(f, axis, -m));
        return s * (R)k.ih[axis];
    }
    __device__ __forceinline__ R lap(const R *f, const FieldCoef &k) const {
        R center = f[g.at(c[0], c[1], c[2])];
        R s = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R sa = (R)k.lap[0] * center;
#pragma unroll
            for (int o = 1; o <= 5; ++o) sa += (R)k.lap[o] * (at(f, a, o) + at(f, a, -o));
            s += sa * (R)k.ih2[a];
        }
        return s;
    }
};

template <typename R>
struct Vec3 {
    const R *p[3];
};

// Neighbours by linear offsets into a padded array whose periodic ghost
// layers (width kGhost >= the stencil reach 5) hold valid images: no index
// wrapping.  Same stencils as Nb.
template <typename R>
struct NbLin {
    int64_t q;      // padded index of the cell
    int64_t s[3];   // strides of x, y, z
    __device__ __forceinline__ R at(const R *f, int axis, int o) const { return f[q + o * s[axis]]; }
    __device__ __forceinline__ R dplus(const R *f, int axis, const FieldCoef &k) const {
        R v = R(0);
#pragma unroll
        for (int m = 1; m <= 3; ++m) v += (R)k.k[m - 1] * (at(f, axis, m) - at(f, axis, 1 - m));
        return v * (R)k.ih[axis];
    }
    __device__ __forceinline__ R dminus(const R *f, int axis, const FieldCoef &k) const {
        R v = R(0);
#pragma unroll
        for (int m = 1; m <= 3; ++m) v += (R)k.k[m - 1] * (at(f, axis, m - 1) - at(f, axis, -m));
        return v * (R)k.ih[axis];
    }
    __device__ __forceinline__ R lap(const R *f, const FieldCoef &k) const {
        R center = f[q];
        R v = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R sa = (R)k.lap[0] * center;
#pragma unroll
            for (int o = 1; o <= 5; ++o) sa += (R)k.lap[o] * (at(f, a, o) + at(f, a, -o));
            v += sa * (R)k.ih2[a];
        }
        return v;
    }
};

template <typename R>
__device__ __forceinline__ NbLin<R> nb_lin(const Geom &g, int i, int j, int k) {
    return NbLin<R>{g.at(i, j, k), {1, (int64_t)g.P[0], (int64_t)g.P[0] * g.P[1]}};
}

// Store v at interior cell (i, j, k) and at every periodic image of it inside
// the ghost layers, so that the array stays readable through NbLin.  Every
// ghost cell is the image of exactly one interior cell.
template <typename R>
__device__ __forceinline__ void store_periodic(R *f, const Geom &g, int i, int j, int k, R v) {
    int x0 = i, y0 = j, z0 = k;
    while (x0 - g.n[0] >= -g.G) x0 -= g.n[0];
    while (y0 - g.n[1] >= -g.G) y0 -= g.n[1];
    while (z0 - g.n[2] >= -g.G) z0 -= g.n[2];
    for (int z = z0; z < g.n[2] + g.G; z += g.n[2])
        for (int y = y0; y < g.n[1] + g.G; y += g.n[1])
            for (int x = x0; x < g.n[0] + g.G; x += g.n[0]) f[g.at(x, y, z)] = v;
}

// Launch shape of the cell kernels below: x along threads, y and z along the
// grid (no division to recover the cell).
constexpr int kCellThreads = 128;
static inline dim3 cell_grid(const Geom &g) {
    return dim3((unsigned)((g.n[0] + kCellThreads - 1) / kCellThreads), (unsigned)g.n[1], (unsigned)g.n[2]);
}

// rhs_a = B_a + alpha beta dt^2 (L B)_a - dt (curl^+ E)_a + alpha dt^2 (curl^+ J)_a
// (eq:EllipticB; the current term's sign follows from eq:bnplus1 + eq:enplus1)
template <typename R>
__global__ void k_rhs(Geom g, FieldCoef k, Vec3<R> E, Vec3<R> B, Vec3<R> J, R *O0, R *O1, R *O2, R ab_dt2,
                      R dt, R a_dt2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    Nb<R> nb{g, {0, 0, 0}};
    unflatten(t, g, nb.c[0], nb.c[1], nb.c[2]);
    int64_t q = g.at(nb.c[0], nb.c[1], nb.c[2]);
    R *out[3] = {O0, O1, O2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        R curlE = nb.dplus(E.p[c], b, k) - nb.dplus(E.p[b], c, k);
        R curlJ = nb.dplus(J.p[c], b, k) - nb.dplus(J.p[b], c, k);
        out[a][q] = B.p[a][q] + ab_dt2 * nb.lap(B.p[a], k) - dt * curlE + a_dt2 * curlJ;
    }
}

// k_rhs for B and E with valid ghost layers (the implicit solver): B and E
// through linear offsets, J (ghosts cleared by the fold) through wrapping.
template <typename R>
__global__ void k_rhs_lin(Geom g, FieldCoef k, Vec3<R> E, Vec3<R> B, Vec3<R> J, R *O0, R *O1, R *O2, R ab_dt2,
                          R dt, R a_dt2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n[0]) return;
    int j = blockIdx.y, kz = blockIdx.z;
    NbLin<R> nl = nb_lin<R>(g, i, j, kz);
    Nb<R> nb{g, {i, j, kz}};
    R *out[3] = {O0, O1, O2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        R curlE = nl.dplus(E.p[c], b, k) - nl.dplus(E.p[b], c, k);
        R curlJ = nb.dplus(J.p[c], b, k) - nb.dplus(J.p[b], c, k);
        out[a][nl.q] = B.p[a][nl.q] + ab_dt2 * nl.lap(B.p[a], k) - dt * curlE + a_dt2 * curlJ;
    }
}

// One Chebyshev sweep (Saad's three-term form, see field_update_impl), plane by
// plane: r = rhs - X + kk L X, X_new = X + c1 (X - X_prev) + c2 r, with each
// component's 31-point Laplacian (NbLin::lap, the same sums in the same order) read
// from a shared xy plane (the block's 32 x 8 nodes and 5 nodes of halo on each
// side) and a register column of the 11 z nodes around the plane.  A block
// marches through kChebZ planes of one component, so every node of X comes
// from L2 or HBM about three times (column, halo, chunk start) instead of 31.
// Planes per block: 8 measured best (C3 beam field update 2.62 ms per step
// against 2.68 at 16 and 2.91 at 32; 3.80 for the node-per-thread sweep that
// read every neighbour through L1/L2).
#ifndef PP_CHEB_Z
#define PP_CHEB_Z 8
#endif
constexpr int kChebBX = 32, kChebBY = 8, kChebZ = PP_CHEB_Z, kChebR = 5;

template <typename R>
__global__ void __launch_bounds__(kChebBX *kChebBY) k_cheb_plane(Geom g, FieldCoef k, Vec3<R> X, Vec3<R> Xp, Vec3<R> Rh,
                                                                 R *O0, R *O1, R *O2, R kk, R c1, R c2, int nzc) {
    __shared__ R pl[kChebBY + 2 * kChebR][kChebBX + 2 * kChebR];
    const int tx = threadIdx.x % kChebBX, ty = threadIdx.x / kChebBX;
    const int x0 = blockIdx.x * kChebBX, y0 = blockIdx.y * kChebBY;
    const int a = blockIdx.z / nzc, zc = blockIdx.z - a * nzc;
    const int z0 = zc * kChebZ, z1 = min(g.n[2], z0 + kChebZ);
    const int i = x0 + tx, j = y0 + ty;
    const bool mine = i < g.n[0] && j < g.n[1];
    // the component's arrays, selected without indexing the parameter arrays
    // at run time (which would copy them to local memory)
    const R *f = a == 0 ? X.p[0] : (a == 1 ? X.p[1] : X.p[2]);
    const R *fp = a == 0 ? Xp.p[0] : (a == 1 ? Xp.p[1] : Xp.p[2]);
    const R *rh = a == 0 ? Rh.p[0] : (a == 1 ? Rh.p[1] : Rh.p[2]);
    R *out = a == 0 ? O0 : (a == 1 ? O1 : O2);
    // Each thread reads at most five x, y positions of the padded array (its
    // column and up to four halo nodes); their plane-0 offsets and whether
    // they lie inside the padded array (every node a computed node reads
    // does) are fixed for the whole march.
    const int64_t ps = (int64_t)g.P[0] * g.P[1];
    auto inside = [&](int x, int y) { return x >= -g.G && x < g.n[0] + g.G && y >= -g.G && y < g.n[1] + g.G; };
    const bool okc = inside(i, j);
    const int64_t qc = okc ? g.at(i, j, 0) : 0;
    const bool okx0 = tx < kChebR && inside(x0 + tx - kChebR, j), okx1 = tx < kChebR && inside(x0 + kChebBX + tx, j);
    const bool oky0 = ty < kChebR && inside(i, y0 + ty - kChebR), oky1 = ty < kChebR && inside(i, y0 + kChebBY + ty);
    const int64_t qx0 = okx0 ? g.at(x0 + tx - kChebR, j, 0) : 0, qx1 = okx1 ? g.at(x0 + kChebBX + tx, j, 0) : 0;
    const int64_t qy0 = oky0 ? g.at(i, y0 + ty - kChebR, 0) : 0, qy1 = oky1 ? g.at(i, y0 + kChebBY + ty, 0) : 0;
    // no periodic image of this column's nodes inside the ghost layers on x or y
    const bool noimg_xy = i >= g.G && i < g.n[0] - g.G && j >= g.G && j < g.n[1] - g.G;
    R col[2 * kChebR + 1];
#pragma unroll
    for (int m = 0; m < 2 * kChebR + 1; ++m) col[m] = okc ? f[qc + (int64_t)(z0 - kChebR + m) * ps] : R(0);
    R lp[kChebR + 1];
#pragma unroll
    for (int o = 0; o <= kChebR; ++o) lp[o] = (R)k.lap[o];
    const R ih2x = (R)k.ih2[0], ih2y = (R)k.ih2[1], ih2z = (R)k.ih2[2];
    // the next plane's halo nodes, rhs and previous iterate are loaded one
    // plane ahead, so that their latency overlaps the current plane's work
    R hx0 = R(0), hx1 = R(0), hy0 = R(0), hy1 = R(0), rhn = R(0), xpn = R(0);
    auto fetch = [&](int z) {
        const int64_t zo = (int64_t)z * ps;
        if (okx0) hx0 = f[qx0 + zo];
        if (okx1) hx1 = f[qx1 + zo];
        if (oky0) hy0 = f[qy0 + zo];
        if (oky1) hy1 = f[qy1 + zo];
        if (mine) {
            rhn = rh[qc + zo];
            xpn = fp[qc + zo];
        }
    };
    fetch(z0);
    for (int z = z0; z < z1; ++z) {
        pl[ty + kChebR][tx + kChebR] = col[kChebR];
        if (tx < kChebR) {
            pl[ty + kChebR][tx] = hx0;
            pl[ty + kChebR][tx + kChebBX + kChebR] = hx1;
        }
        if (ty < kChebR) {
            pl[ty][tx + kChebR] = hy0;
            pl[ty + kChebBY + kChebR][tx + kChebR] = hy1;
        }
        const R rhz = rhn, xpz = xpn;
        __syncthreads();
        if (z + 1 < z1) fetch(z + 1);
        if (mine) {
            const R center = col[kChebR];
            R v = R(0);
            R sa = lp[0] * center;
#pragma unroll
            for (int o = 1; o <= kChebR; ++o)
                sa += lp[o] * (pl[ty + kChebR][tx + kChebR + o] + pl[ty + kChebR][tx + kChebR - o]);
            v += sa * ih2x;
            sa = lp[0] * center;
#pragma unroll
            for (int o = 1; o <= kChebR; ++o)
                sa += lp[o] * (pl[ty + kChebR + o][tx + kChebR] + pl[ty + kChebR - o][tx + kChebR]);
            v += sa * ih2y;
            sa = lp[0] * center;
#pragma unroll
            for (int o = 1; o <= kChebR; ++o) sa += lp[o] * (col[kChebR + o] + col[kChebR - o]);
            v += sa * ih2z;
            const R x = center;
            const R r = rhz - x + kk * v;
            const R nv = x + c1 * (x - xpz) + c2 * r;
            if (noimg_xy && z >= g.G && z < g.n[2] - g.G)
                out[qc + (int64_t)z * ps] = nv;
            else
                store_periodic(out, g, i, j, z, nv);
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 2 * kChebR; ++m) col[m] = col[m + 1];
        if (z + 1 < z1 && okc) col[2 * kChebR] = f[qc + (int64_t)(z + 1 + kChebR) * ps];
    }
}

// k_e_update with Bn and Bo ghost-valid (linear offsets).
template <typename R>
__global__ void k_e_update_lin(Geom g, FieldCoef k, R *E0, R *E1, R *E2, Vec3<R> Bn, Vec3<R> Bo, Vec3<R> J, R alpha,
                               R beta, R dt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n[0]) return;
    int j = blockIdx.y, kz = blockIdx.z;
    NbLin<R> nl = nb_lin<R>(g, i, j, kz);
    R *E[3] = {E0, E1, E2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        R cur = alpha * (nl.dminus(Bn.p[c], b, k) - nl.dminus(Bn.p[b], c, k)) +
                beta * (nl.dminus(Bo.p[c], b, k) - nl.dminus(Bo.p[b], c, k));
        E[a][nl.q] = E[a][nl.q] + dt * (cur - J.p[a][nl.q]);
    }
}

// E_new = E + dt (curl^- (alpha B_new + beta B_old) - J)   (eq:enplus1, c^2 mu0 = 1)
template <typename R>
struct MixB {
    const R *Bn, *Bo;
    R al, be;
};

template <typename R>
__global__ void k_e_update(Geom g, FieldCoef k, R *E0, R *E1, R *E2, Vec3<R> Bn, Vec3<R> Bo, Vec3<R> J, R alpha,
                           R beta, R dt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    Nb<R> nb{g, {0, 0, 0}};
    unflatten(t, g, nb.c[0], nb.c[1], nb.c[2]);
    int64_t q = g.at(nb.c[0], nb.c[1], nb.c[2]);
    R *E[3] = {E0, E1, E2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        R cur = alpha * (nb.dminus(Bn.p[c], b, k) - nb.dminus(Bn.p[b], c, k)) +
                beta * (nb.dminus(Bo.p[c], b, k) - nb.dminus(Bo.p[b], c, k));
        E[a][q] = E[a][q] + dt * (cur - J.p[a][q]);
    }
}

// Periodic ghost fill of E (from its own interior) and B (from src, which may
// be a different array than B: the converged relaxation iterate).
template <typename R>
__global__ void k_ghost_fill(Geom g, R *E0, R *E1, R *E2, const R *S0, const R *S1, const R *S2, R *B0, R *B1, R *B2,
                             int e_ghost_only) {
    int64_t total = g.padded_size();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i = (int)(t % g.P[0]);
    int64_t r = t / g.P[0];
    int j = (int)(r % g.P[1]);
    int k = (int)(r / g.P[1]);
    int ci = i - g.G, cj = j - g.G, ck = k - g.G;
    bool ghost = ci < 0 || cj < 0 || ck < 0 || ci >= g.n[0] || cj >= g.n[1] || ck >= g.n[2];
    int64_t src = g.at(wrap(ci, g.n[0]), wrap(cj, g.n[1]), wrap(ck, g.n[2]));
    if (ghost || !e_ghost_only) {
        E0[t] = E0[src]; E1[t] = E1[src]; E2[t] = E2[src];
    }
    B0[t] = S0[src]; B1[t] = S1[src]; B2[t] = S2[src];
}

template <typename R>
static Vec3<R> v3(void *const p[3]) {
    return Vec3<R>{{(const R *)p[0], (const R *)p[1], (const R *)p[2]}};
}

static FieldCoef field_coef(const Ctx &c) {
    FieldCoef k;
    double h[3] = {c.d.dx, c.d.dy, c.d.dz};
    for (int m = 0; m < 3; ++m) k.k[m] = c.fd[m];
    for (int m = 0; m < 6; ++m) k.lap[m] = c.lap[m];
    for (int a = 0; a < 3; ++a) {
        k.ih[a] = 1.0 / h[a];
        k.ih2[a] = 1.0 / (h[a] * h[a]);
    }
    return k;
}

template <typename R>
static cudaError_t field_update_impl(Ctx &c) {
    const Geom &g = c.g;
    FieldCoef k = field_coef(c);
    // dt of this solve: the step, or the drift of a 4th-order substep
    double al = c.d.alpha, be = 1.0 - c.d.alpha, dt = c.drift_dt;
    double kk = al * al * dt * dt;
    const Ctx::Cheb &ch = c.cheb[c.cheb_sel];
    cudaError_t e;
    // B and E arrive with valid ghost layers (every writer of them fills
    // them), and each sweep writes its iterate with ghosts: the stencils read
    // through linear offsets.
    const dim3 cg = cell_grid(g);
    k_rhs_lin<R><<<cg, kCellThreads, 0, c.st>>>(g, k, v3<R>(c.E), v3<R>(c.B), v3<R>(c.J), (R *)c.R[0], (R *)c.R[1],
                                                (R *)c.R[2], (R)(al * be * dt * dt), (R)dt, (R)(al * dt * dt));
    ++c.nlaunch;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Chebyshev semi-iteration on the spectrum [1, lmax] of the SPD operator,
    // starting from B^n (Saad, Iterative Methods, Alg. 12.1 in 3-term form).
    double theta = ch.theta, delta = ch.delta;
    const int nzc = (g.n[2] + kChebZ - 1) / kChebZ;
    const dim3 pg((unsigned)((g.n[0] + kChebBX - 1) / kChebBX), (unsigned)((g.n[1] + kChebBY - 1) / kChebBY),
                  (unsigned)(3 * nzc));
    void **cur = c.B, **prev = c.B;
    void **bufs[2] = {c.Xa, c.Xb};
    int nb = 0;
    double rho_prev = delta > 0 ? delta / theta : 0.0;
    for (int it = 0; it < ch.iters; ++it) {
        double c1, c2;
        if (it == 0) {
            c1 = 0.0;
            c2 = 1.0 / theta;
        } else {
            double sigma = theta / delta;
            double rho = 1.0 / (2.0 * sigma - rho_prev);
            c1 = rho * rho_prev;
            c2 = 2.0 * rho / delta;
            rho_prev = rho;
        }
        // output: a scratch buffer that is neither cur nor (when prev is B) B
        void **out = (prev == c.B || prev == cur) ? bufs[nb] : prev;
        if (out == cur) out = bufs[1 - nb];
        k_cheb_plane<R><<<pg, kChebBX * kChebBY, 0, c.st>>>(g, k, v3<R>(cur), v3<R>(prev), v3<R>(c.R),
                                                             (R *)out[0], (R *)out[1], (R *)out[2], (R)kk, (R)c1,
                                                             (R)c2, nzc);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        prev = cur;
        cur = out;
        nb = (out == bufs[0]) ? 1 : 0;
    }
    c.last_iters = ch.iters;
    c.last_kk = kk;
    c.filtered_after_solve = false;
    // eq:enplus1 with B^{n+1} = cur, B^n = B
    k_e_update_lin<R><<<cg, kCellThreads, 0, c.st>>>(g, k, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], v3<R>(cur),
                                                     v3<R>(c.B), v3<R>(c.J), (R)al, (R)be, (R)dt);
    ++c.nlaunch;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned pblocks = (unsigned)((g.padded_size() + 255) / 256);
    k_ghost_fill<R><<<pblocks, 256, 0, c.st>>>(g, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], (const R *)cur[0],
                                               (const R *)cur[1], (const R *)cur[2], (R *)c.B[0], (R *)c.B[1],
                                               (R *)c.B[2], 1);
    ++c.nlaunch;
    return cudaGetLastError();
}

// Explicit FDTD variant (the cold-beam comparison of Sec. VIII): Yee's
// leap-frog with the same staggered differences, B in two half steps so that
// E and B stay at one time level:
//   B^{n+1/2} = B^n - dt/2 curl^+ E^n,  E^{n+1} = E^n + dt (curl^- B^{n+1/2} - J),
//   B^{n+1} = B^{n+1/2} - dt/2 curl^+ E^{n+1}.
// The half steps are k_rhs with alpha = 0, the full step k_e_update with
// alpha = 1.
template <typename R>
static cudaError_t field_update_explicit_impl(Ctx &c) {
    const Geom &g = c.g;
    FieldCoef k = field_coef(c);
    unsigned blocks = (unsigned)((g.cells() + 255) / 256);
    unsigned pblocks = (unsigned)((g.padded_size() + 255) / 256);
    const R half = (R)(0.5 * c.drift_dt);
    cudaError_t e;
    for (int pass = 0; pass < 2; ++pass) {
        // B half step into the scratch R, then B := R with its ghost layers
        k_rhs<R><<<blocks, 256, 0, c.st>>>(g, k, v3<R>(c.E), v3<R>(c.B), v3<R>(c.J), (R *)c.R[0], (R *)c.R[1],
                                           (R *)c.R[2], (R)0, half, (R)0);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_ghost_fill<R><<<pblocks, 256, 0, c.st>>>(g, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], (const R *)c.R[0],
                                                   (const R *)c.R[1], (const R *)c.R[2], (R *)c.B[0], (R *)c.B[1],
                                                   (R *)c.B[2], 1);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (pass == 1) break;
        // E full step with B^{n+1/2}, then E's ghost layers (B copies onto itself)
        k_e_update<R><<<blocks, 256, 0, c.st>>>(g, k, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], v3<R>(c.B), v3<R>(c.B),
                                                v3<R>(c.J), (R)1, (R)0, (R)c.drift_dt);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_ghost_fill<R><<<pblocks, 256, 0, c.st>>>(g, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], (const R *)c.B[0],
                                                   (const R *)c.B[1], (const R *)c.B[2], (R *)c.B[0], (R *)c.B[1],
                                                   (R *)c.B[2], 1);
        ++c.nlaunch;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    c.last_iters = 0;   // no relaxation
    c.last_kk = 0.0;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Divergence filter (the paper's divergence cleaning of E for the direct
// current, and the periodic filter of E and B in long FP32 runs): each pass is
// one simultaneous smoothing step
//   E += tau grad^+ (div^- E - rho),   B += tau grad^- (div^+ B),
// tau = 1 / max(sum_a K_a^2), which removes the Nyquist-scale error in one
// pass and damps every other non-constant mode.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_div_error(Geom g, FieldCoef k, Vec3<R> F, const double *rho, int plus, R *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    Nb<R> nb{g, {0, 0, 0}};
    unflatten(t, g, nb.c[0], nb.c[1], nb.c[2]);
    R d = plus ? nb.dplus(F.p[0], 0, k) + nb.dplus(F.p[1], 1, k) + nb.dplus(F.p[2], 2, k)
               : nb.dminus(F.p[0], 0, k) + nb.dminus(F.p[1], 1, k) + nb.dminus(F.p[2], 2, k);
    out[g.at(nb.c[0], nb.c[1], nb.c[2])] = rho ? d - (R)rho[t] : d;
}

template <typename R>
__global__ void k_grad_add(Geom g, FieldCoef k, const R *r, R *F0, R *F1, R *F2, R tau, int plus) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    Nb<R> nb{g, {0, 0, 0}};
    unflatten(t, g, nb.c[0], nb.c[1], nb.c[2]);
    int64_t q = g.at(nb.c[0], nb.c[1], nb.c[2]);
    R *F[3] = {F0, F1, F2};
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a][q] += tau * (plus ? nb.dplus(r, a, k) : nb.dminus(r, a, k));
}

template <typename R>
static cudaError_t divergence_filter_impl(Ctx &c) {
    cudaError_t e = launch_rho(c);   // rho at the particles' current positions
    if (e != cudaSuccess) return e;
    const Geom &g = c.g;
    FieldCoef k = field_coef(c);
    unsigned blocks = (unsigned)((g.cells() + 255) / 256);
    const R tau = (R)c.filter_tau;
    // scratch: the relaxation iterates (free after a solve); the solve's
    // right-hand side in R stays for the residual diagnostics
    R *eE = (R *)c.Xa[0], *eB = (R *)c.Xa[1];
    for (int p = 0; p < c.filter_passes; ++p) {
        k_div_error<R><<<blocks, 256, 0, c.st>>>(g, k, v3<R>(c.E), c.rho, 0, eE);
        k_grad_add<R><<<blocks, 256, 0, c.st>>>(g, k, eE, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], tau, 1);
        k_div_error<R><<<blocks, 256, 0, c.st>>>(g, k, v3<R>(c.B), nullptr, 1, eB);
        k_grad_add<R><<<blocks, 256, 0, c.st>>>(g, k, eB, (R *)c.B[0], (R *)c.B[1], (R *)c.B[2], tau, 0);
        c.nlaunch += 4;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    unsigned pblocks = (unsigned)((g.padded_size() + 255) / 256);
    k_ghost_fill<R><<<pblocks, 256, 0, c.st>>>(g, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], (const R *)c.B[0],
                                               (const R *)c.B[1], (const R *)c.B[2], (R *)c.B[0], (R *)c.B[1],
                                               (R *)c.B[2], 1);
    ++c.nlaunch;
    c.filtered_after_solve = true;   // B moved since the last solve: its residual no longer measures it
    return cudaGetLastError();
}

cudaError_t launch_divergence_filter(Ctx &c) {
    return c.fp64 ? divergence_filter_impl<double>(c) : divergence_filter_impl<float>(c);
}

cudaError_t launch_field_update(Ctx &c) {
    if (c.field_solver == PP_FIELD_EXPLICIT)
        return c.fp64 ? field_update_explicit_impl<double>(c) : field_update_explicit_impl<float>(c);
    return c.fp64 ? field_update_impl<double>(c) : field_update_impl<float>(c);
}

template <typename R>
static cudaError_t ghost_fill_impl(Ctx &c, void *const sE[3], void *const sB[3]) {
    (void)sE;
    unsigned pblocks = (unsigned)((c.g.padded_size() + 255) / 256);
    k_ghost_fill<R><<<pblocks, 256, 0, c.st>>>(c.g, (R *)c.E[0], (R *)c.E[1], (R *)c.E[2], (const R *)sB[0],
                                               (const R *)sB[1], (const R *)sB[2], (R *)c.B[0], (R *)c.B[1],
                                               (R *)c.B[2], 1);
    ++c.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_ghost_fill(Ctx &c, void *const sE[3], void *const sB[3]) {
    return c.fp64 ? ghost_fill_impl<double>(c, sE, sB) : ghost_fill_impl<float>(c, sE, sB);
}

// ---------------------------------------------------------------------------
// FP64 mesh diagnostics: sums (energies, charge) and maxima (|rho|, Gauss
// residual, its drift from G_0, div B, relaxation residual, |rhs|).
// ---------------------------------------------------------------------------
constexpr int kDiagSums = 4, kDiagMax = 6, kDiagN = kDiagSums + kDiagMax;

template <typename R>
__global__ void k_mesh_diag(Geom g, FieldCoef k, Vec3<R> E, Vec3<R> B, Vec3<R> Rh, const double *rho, double *G0,
                            int capture, double kk, double *partial) {
    double v[kDiagN];
    for (int m = 0; m < kDiagN; ++m) v[m] = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.cells(); t += (int64_t)gridDim.x * blockDim.x) {
        Nb<R> nb{g, {0, 0, 0}};
        unflatten(t, g, nb.c[0], nb.c[1], nb.c[2]);
        int64_t q = g.at(nb.c[0], nb.c[1], nb.c[2]);
        double e0 = E.p[0][q], e1 = E.p[1][q], e2 = E.p[2][q];
        double b0 = B.p[0][q], b1 = B.p[1][q], b2 = B.p[2][q];
        v[0] += 0.5 * (e0 * e0 + e1 * e1 + e2 * e2);
        v[1] += 0.5 * (b0 * b0 + b1 * b1 + b2 * b2);
        v[2] += 0.5 * e0 * e0;
        double r = rho[t];
        v[3] += r;
        double divE = 0.0, divB = 0.0;
        for (int a = 0; a < 3; ++a) {
            divE += (double)nb.dminus(E.p[a], a, k);
            divB += (double)nb.dplus(B.p[a], a, k);
        }
        double G = divE - r;
        if (capture) G0[t] = G;
        v[4] = fmax(v[4], fabs(r));
        v[5] = fmax(v[5], fabs(G));
        v[6] = fmax(v[6], fabs(G - G0[t]));
        v[7] = fmax(v[7], fabs(divB));
        for (int a = 0; a < 3; ++a) {
            double res = (double)Rh.p[a][q] - ((double)B.p[a][q] - kk * (double)nb.lap(B.p[a], k));
            v[8] = fmax(v[8], fabs(res));
            v[9] = fmax(v[9], fabs((double)Rh.p[a][q]));
        }
    }
    __shared__ double sh[kDiagN][256];
    for (int m = 0; m < kDiagN; ++m) sh[m][threadIdx.x] = v[m];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int m = 0; m < kDiagN; ++m) {
                double a = sh[m][threadIdx.x], b = sh[m][threadIdx.x + s];
                sh[m][threadIdx.x] = m < kDiagSums ? a + b : fmax(a, b);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int m = 0; m < kDiagN; ++m) partial[(int64_t)blockIdx.x * kDiagN + m] = sh[m][0];
}

__global__ void k_diag_final(const double *partial, int nblk, double *out) {
    int m = threadIdx.x;
    if (m >= kDiagN) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) {
        double v = partial[(int64_t)b * kDiagN + m];
        acc = m < kDiagSums ? acc + v : fmax(acc, v);
    }
    out[m] = acc;
}

constexpr int kDiagBlocks = 512;

template <typename R>
static cudaError_t mesh_diag_impl(Ctx &c, double *host_out) {
    FieldCoef k = field_coef(c);
    int capture = c.have_G0 ? 0 : 1;
    double kk = c.last_kk;   // residual of the last solve
    int64_t want = (c.g.cells() + 255) / 256;
    int nblk = (int)(want < kDiagBlocks ? want : kDiagBlocks);
    k_mesh_diag<R><<<nblk, 256, 0, c.st>>>(c.g, k, v3<R>(c.E), v3<R>(c.B), v3<R>(c.R), c.rho, c.G0, capture, kk, c.d_red);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, 32, 0, c.st>>>(c.d_red, nblk, c.d_out);
    c.nlaunch += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaMemcpyAsync(host_out, c.d_out, sizeof(double) * kDiagN, cudaMemcpyDeviceToHost, c.st);
    if (e != cudaSuccess) return e;
    c.have_G0 = true;
    return cudaSuccess;
}

cudaError_t launch_mesh_diag(Ctx &c, double *host_out) {
    return c.fp64 ? mesh_diag_impl<double>(c, host_out) : mesh_diag_impl<float>(c, host_out);
}

}  // namespace pp
