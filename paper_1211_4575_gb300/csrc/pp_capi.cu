// pp_capi.cu -- the C ABI of include/pp.h: context lifecycle, loading and
// unloading, the step driver (Sec. III step order 1-5), diagnostics and
// checkpointing.  All device work goes through the kernels of pp_particles.cu,
// pp_mesh.cu and pp_sort.cu on the context's stream; no step of the particle
// or field update runs on the host.
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pp_ctx.cuh"
#include "pp_tma.cuh"

// NVTX range over a host scope: each phase of a step shows up by name in a
// profiler timeline (ncu --nvtx, Nsight Systems).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

using namespace pp;

static char g_last_error[512] = "";

static int fail(Ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
static int fail(Ctx *c, int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    char *dst = c ? c->err : g_last_error;
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CU(expr)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess) return fail(c, PP_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// Setup of the constant operators
// ---------------------------------------------------------------------------
static void fd_coeffs(int order, double k[3]) {
    // Staggered first-derivative coefficients (Sec. III).  6th order: the
    // printed a = 25/21 violates a + 3b + 5c = 1; a = 75/64 is the value that
    // satisfies the Taylor conditions with the printed b and c.
    if (order == 6) { k[0] = 75.0 / 64.0; k[1] = -25.0 / 384.0; k[2] = 3.0 / 640.0; }
    else if (order == 4) { k[0] = 9.0 / 8.0; k[1] = -1.0 / 24.0; k[2] = 0.0; }
    else { k[0] = 1.0; k[1] = 0.0; k[2] = 0.0; }
}

// First row g of the inverse of the symmetric circulant line operator with
// symbol p(th) = (a+b+c) + 2(b+c) cos th + 2c cos 2th (n points), via its
// discrete Fourier representation.
static void circulant_inverse(int n, const double k[3], std::vector<double> &g) {
    double d0 = k[0] + k[1] + k[2], d1 = k[1] + k[2], d2 = k[2];
    g.assign(n, 0.0);
    for (int m = 0; m < n; ++m) {
        double th = 2.0 * M_PI * m / n;
        double inv = 1.0 / (d0 + 2.0 * d1 * cos(th) + 2.0 * d2 * cos(2.0 * th));
        for (int q = 0; q < n; ++q) g[q] += cos(th * q) * inv;
    }
    for (int q = 0; q < n; ++q) g[q] /= n;
}

// Drift (a) and kick (b) fractions of the four substeps of the symmetric
// fourth-order integrator (Sec. III; Forest & Ruth 1990, Candy & Rozmus
// 1991): kick b_i dt, then drift a_i dt, so that every kick is centred on the
// position time.  w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3) w1.
static void step4_fractions(double a[4], double b[4]) {
    const double r = cbrt(2.0);
    const double w1 = 1.0 / (2.0 - r), w0 = -r * w1;
    a[0] = a[3] = 0.5 * w1;
    a[1] = a[2] = 0.5 * (w0 + w1);
    b[0] = 0.0;
    b[1] = b[3] = w1;
    b[2] = w0;
}

// Chebyshev bounds of A = 1 - alpha^2 dt^2 L (spectrum in [1, 1 + kk sum_a
// max K_a^2]) and the iteration count that reaches relax_tol.
static void cheb_setup(const Ctx *c, double dt, Ctx::Cheb &out) {
    double h[3] = {c->d.dx, c->d.dy, c->d.dz};
    double kk = c->d.alpha * c->d.alpha * dt * dt;
    double lmax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double best = 0.0;
        for (int s = 0; s <= 4000; ++s) {
            double th = M_PI * s / 4000.0;
            double K = 2.0 * (c->fd[0] * sin(0.5 * th) + c->fd[1] * sin(1.5 * th) + c->fd[2] * sin(2.5 * th));
            best = fmax(best, K * K);
        }
        lmax += kk * best * 1.0005 / (h[a] * h[a]);
    }
    out.theta = 0.5 * (lmax + 1.0);
    out.delta = 0.5 * (lmax - 1.0);
    double sk = sqrt(lmax);
    double rho = (sk - 1.0) / (sk + 1.0);
    double target = c->d.relax_tol / sqrt(3.0 * (double)c->g.cells()) / sk;
    int it = 1;
    if (out.delta > 0.0) {
        double rk = rho;
        while (it < 10000 && 2.0 * rk / (1.0 + rk * rk) > target) {
            rk *= rho;
            ++it;
        }
    }
    out.iters = it < c->d.relax_max_iter ? it : c->d.relax_max_iter;
}

static int setup_operators(Ctx *c) {
    fd_coeffs(c->d.field_order, c->fd);
    // 1D stencil of d^+ d^-: autocorrelation of the half-offset kernel
    // t(+-(m-1/2)) = +-k_m
    double t[6] = {-c->fd[2], -c->fd[1], -c->fd[0], c->fd[0], c->fd[1], c->fd[2]};
    for (int s = 0; s <= 5; ++s) {
        double acc = 0.0;
        for (int p = 0; p < 6; ++p) {
            int q = p + s;   // offsets differ by s
            if (q < 6) acc += t[q] * t[p];
        }
        c->lap[s] = -acc;    // l_s = sum_p t_p t_{s-p} = -sum_p t_{p+s} t_p by antisymmetry
    }
    // high-order current taps
    std::vector<double> host(3 * kMaxTaps, 0.0);
    double eps = c->fp64 ? 1e-18 : 1e-10;
    for (int a = 0; a < 3; ++a) {
        c->ntaps[a] = 0;
        if (c->d.field_order == 2) continue;
        int n = c->g.n[a];
        std::vector<double> gi;
        circulant_inverse(n, c->fd, gi);
        if (n <= kMaxTaps) {
            c->full_circ[a] = true;
            c->ntaps[a] = n;
            for (int m = 0; m < n; ++m) host[a * kMaxTaps + m] = gi[m];
        } else {
            int K = 1;
            while (K < n / 2 && K < (kMaxTaps - 1) / 2 && fabs(gi[K + 1]) > eps * fabs(gi[0])) ++K;
            c->full_circ[a] = false;
            c->ntaps[a] = 2 * K + 1;
            for (int m = 0; m <= 2 * K; ++m) host[a * kMaxTaps + m] = gi[abs(m - K)];
        }
    }
    cudaError_t e = cudaMalloc(&c->taps, sizeof(double) * 3 * kMaxTaps);
    if (e != cudaSuccess) return fail(c, PP_ECUDA, "taps: %s", cudaGetErrorString(e));
    e = cudaMemcpy(c->taps, host.data(), sizeof(double) * 3 * kMaxTaps, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(c, PP_ECUDA, "taps copy: %s", cudaGetErrorString(e));
    // Chebyshev bounds of A = 1 - alpha^2 dt^2 L for every solve step the
    // context takes: the step dt and the drifts of the 4th-order substeps
    double a[4], b[4];
    step4_fractions(a, b);
    const double dts[3] = {c->d.dt, fabs(a[0]) * c->d.dt, fabs(a[1]) * c->d.dt};
    for (int q = 0; q < 3; ++q) cheb_setup(c, dts[q], c->cheb[q]);
    c->cheb_sel = 0;
    c->kick_dt = c->drift_dt = c->d.dt;
    // divergence filter step: 1 / max over wave numbers of sum_a K_a^2
    {
        double h[3] = {c->d.dx, c->d.dy, c->d.dz}, lam = 0.0;
        for (int a = 0; a < 3; ++a) {
            double best = 0.0;
            for (int s = 0; s <= 4000; ++s) {
                double th = M_PI * s / 4000.0;
                double K = 2.0 * (c->fd[0] * sin(0.5 * th) + c->fd[1] * sin(1.5 * th) + c->fd[2] * sin(2.5 * th));
                best = fmax(best, K * K);
            }
            lam += best / (h[a] * h[a]);
        }
        c->filter_tau = 1.0 / lam;
    }
    c->last_kk = c->d.alpha * c->d.alpha * c->d.dt * c->d.dt;
    return PP_OK;
}

// ---------------------------------------------------------------------------
// Lifecycle
// ---------------------------------------------------------------------------
extern "C" int pp_init_grid(pp_ctx **out, const pp_grid_desc *d) {
    Ctx *c = nullptr;
    if (!out || !d) return fail(c, PP_EINVAL, "pp_init_grid: NULL argument");
    *out = nullptr;
    const int bnd[3] = {d->boundary_x, d->boundary_y, d->boundary_z};
    const int nphys[3] = {d->nx, d->ny, d->nz};
    bool walls[3];
    int n[3];   // mesh cells: the mirror-extended box (twice the cells) on walled axes
    for (int a = 0; a < 3; ++a) {
        if (bnd[a] != PP_BOUNDARY_PERIODIC && bnd[a] != PP_BOUNDARY_WALLS)
            return fail(c, PP_EINVAL, "unknown boundary %d on axis %d", bnd[a], a);
        walls[a] = bnd[a] == PP_BOUNDARY_WALLS;
        if (nphys[a] < 1) return fail(c, PP_EINVAL, "grid size %d on axis %d below 1", nphys[a], a);
        n[a] = walls[a] ? 2 * nphys[a] : nphys[a];
    }
    double h[3] = {d->dx, d->dy, d->dz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || n[a] > 1023)
            return fail(c, PP_EINVAL, "grid size %d on axis %d outside [1, 1023]%s", n[a], a,
                        walls[a] ? " (between walls the mesh holds twice the cells)" : "");
        if (!(h[a] > 0.0)) return fail(c, PP_EINVAL, "cell size on axis %d must be > 0", a);
        if (!(d->dt > 0.0) || !(d->dt / h[a] < 1.0))
            return fail(c, PP_EINVAL, "need 0 < c dt / d < 1 on every axis (axis %d: %g)", a, d->dt / h[a]);
    }
    {
        // int32 sort keys: tile-padded cells times the octant sub-keys must stay below 2^31
        int64_t padded = 1;
        for (int a = 0; a < 3; ++a) padded *= (int64_t)((n[a] + 7) / 8 * 8);
        if (padded * kSubKeys >= ((int64_t)1 << 31))
            return fail(c, PP_EINVAL, "grid of %lld (tile-padded) cells above the 2^28 limit", (long long)padded);
    }
    if (d->c != 1.0 || d->eps0 != 1.0) return fail(c, PP_EINVAL, "the library is normalised to c = eps0 = 1");
    if (d->field_order != 2 && d->field_order != 4 && d->field_order != 6)
        return fail(c, PP_EINVAL, "field_order must be 2, 4 or 6");
    if (!(d->alpha >= 0.5 && d->alpha < 1.0)) return fail(c, PP_EINVAL, "alpha must lie in [0.5, 1)");
    if (d->shape_order < 1 || d->shape_order > 3) return fail(c, PP_EINVAL, "shape_order must be 1, 2 or 3");
    if (d->pusher != PP_VAY && d->pusher != PP_BORIS) return fail(c, PP_EINVAL, "unknown pusher");
    if (d->precision != PP_FP64 && d->precision != PP_MIXED32) return fail(c, PP_EINVAL, "unknown precision");
    if (d->relax_max_iter < 1 || !(d->relax_tol > 0.0)) return fail(c, PP_EINVAL, "relaxation cap and tolerance must be > 0");
    if (d->sort_interval < 0) return fail(c, PP_EINVAL, "sort_interval must be >= 0");
    if (d->deposit_mode < 0 || d->deposit_mode > 3) return fail(c, PP_EINVAL, "unknown deposit_mode");
    const bool tiled_mode = d->deposit_mode == PP_DEPOSIT_TILED || d->deposit_mode == PP_DEPOSIT_CELLS;
    if (tiled_mode && d->precision != PP_MIXED32)
        return fail(c, PP_EINVAL, "the tiled deposits exist for PP_MIXED32 only");
    if (tiled_mode && (n[0] % 8 || n[1] % 8 || n[2] % 8))
        return fail(c, PP_EINVAL, "the tiled deposits need every mesh size to be a multiple of 8%s",
                    (walls[0] || walls[1] || walls[2]) ? " (twice the cells on a walled axis)" : "");

    pp_ctx *p = new (std::nothrow) pp_ctx();
    if (!p) return fail(c, PP_ENOMEM, "host allocation failed");
    c = p;
    c->d = *d;
    c->st = (cudaStream_t)d->stream;
    c->fp64 = d->precision == PP_FP64;
    c->rsz = c->fp64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) c->wall[a] = walls[a] ? nphys[a] : 0;
    for (int a = 0; a < 3; ++a) {
        c->g.n[a] = n[a];
        c->g.P[a] = n[a] + 2 * kGhost;
    }
    c->g.G = kGhost;
    int64_t P = c->g.padded_size();
    size_t bytes = (size_t)P * c->rsz;
    cudaError_t e = cudaMalloc(&c->mesh, bytes * 21);
    if (e != cudaSuccess) {
        int r = fail(nullptr, PP_ENOMEM, "mesh allocation (%zu bytes): %s", bytes * 21, cudaGetErrorString(e));
        delete p;
        return r;
    }
    char *m = (char *)c->mesh;
    void **groups[7] = {c->E, c->B, c->J, c->Jt, c->R, c->Xa, c->Xb};
    for (int gidx = 0; gidx < 7; ++gidx)
        for (int a = 0; a < 3; ++a) groups[gidx][a] = m + (size_t)(gidx * 3 + a) * bytes;
    int rc = PP_OK;
    auto chk = [&](cudaError_t ee, const char *what) {
        if (ee != cudaSuccess && rc == PP_OK) rc = fail(c, PP_ECUDA, "%s: %s", what, cudaGetErrorString(ee));
    };
    chk(cudaMemset(c->mesh, 0, bytes * 21), "mesh clear");
    chk(cudaMalloc(&c->rho, sizeof(double) * c->g.cells()), "rho");
    chk(cudaMalloc(&c->G0, sizeof(double) * c->g.cells()), "G0");
    if (rc == PP_OK) chk(cudaMemset(c->G0, 0, sizeof(double) * c->g.cells()), "G0 clear");
    chk(cudaMalloc(&c->d_status, sizeof(int)), "status");
    if (rc == PP_OK) chk(cudaMemset(c->d_status, 0, sizeof(int)), "status clear");
    chk(cudaMallocHost(&c->h_status, sizeof(int)), "status mirror");
    chk(cudaMallocHost(&c->h_count, sizeof(int32_t)), "count mirror");
    chk(cudaMalloc(&c->d_red, sizeof(double) * 512 * 16), "reduction partials");
    chk(cudaMalloc(&c->d_out, sizeof(double) * (16 + PP_MAX_SPECIES)), "reduction results");
    chk(cudaMalloc(&c->d_nslow, sizeof(unsigned long long)), "fallback counter");
    chk(cudaMalloc(&c->d_slow_count, sizeof(unsigned) * PP_MAX_SPECIES), "fallback lists");
    if (rc == PP_OK) chk(cudaMemset(c->d_nslow, 0, sizeof(unsigned long long)), "fallback counter clear");
    if (rc == PP_OK) chk(sort_setup(*c), "sort setup");
    if (rc == PP_OK) rc = setup_operators(c);
    if (rc != PP_OK) {
        snprintf(g_last_error, sizeof g_last_error, "%s", c->err);
        pp_destroy(p);
        return rc;
    }
    *out = p;
    if (d->alpha < 0.525 && d->field_order == 6 && d->shape_order == 3)
        return fail(c, PP_WSTAB, "alpha %.4g < 0.525 with 6th-order fields and PCS is reported unstable", d->alpha);
    return PP_OK;
}

// Drop every captured step graph (their launch arguments no longer hold).
static void graphs_clear(Ctx *c) {
    for (int q = 0; q < kGraphSlots; ++q) {
        if (c->graphs[q].exec) cudaGraphExecDestroy(c->graphs[q].exec);
        c->graphs[q] = StepGraph();
    }
    c->graph_next = 0;
}

extern "C" int pp_destroy(pp_ctx *p) {
    if (!p) return PP_OK;
    Ctx *c = p;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    graphs_clear(c);
    for (int s = 0; s < c->nspecies; ++s) {
        cudaFree(c->sp[s].buf);
        cudaFree(c->sp[s].alt);
        cudaFree(c->sp[s].keys);
        cudaFree(c->sp[s].perm);
        cudaFree(c->sp[s].cell_start);
    }
    cudaFree(c->mesh);
    cudaFree(c->rho);
    cudaFree(c->G0);
    cudaFree(c->taps);
    cudaFree(c->counts);
    cudaFree(c->scan_tmp);
    cudaFree(c->d_status);
    cudaFree(c->d_red);
    cudaFree(c->d_out);
    cudaFree(c->d_nslow);
    cudaFree(c->d_slow_count);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_count) cudaFreeHost(c->h_count);
    for (int q = 0; q < c->prof_cap; ++q) {
        cudaEventDestroy(c->prof_ev[q].a);
        cudaEventDestroy(c->prof_ev[q].b);
    }
    free(c->prof_ev);
    delete p;
    return PP_OK;
}

extern "C" const char *pp_last_error(const pp_ctx *p) { return p ? p->err : g_last_error; }

extern "C" int pp_init_species(pp_ctx *p, const pp_species_desc *sd, int *sid) {
    Ctx *c = p;
    if (!c || !sd || !sid) return fail(c, PP_EINVAL, "pp_init_species: NULL argument");
    if (c->nspecies >= PP_MAX_SPECIES) return fail(c, PP_EINVAL, "at most %d species", PP_MAX_SPECIES);
    if (!(sd->m > 0.0) || !isfinite(sd->q) || !isfinite(sd->w) || sd->capacity < 0)
        return fail(c, PP_EINVAL, "species needs m > 0, finite q and w, capacity >= 0");
    if (sd->capacity > (int64_t)0x7fffffff - 64) return fail(c, PP_EINVAL, "capacity above 2^31 - 64");
    Species &S = c->sp[c->nspecies];
    S = Species();
    S.q = sd->q;
    S.m = sd->m;
    S.w = sd->w;
    S.limit = sd->capacity;
    S.cap = (sd->capacity + 63) / 64 * 64;
    if (S.cap == 0) S.cap = 64;
    size_t per = c->fp64 ? 6 * sizeof(double) : sizeof(int32_t) + 6 * sizeof(float);
    size_t bytes = per * (size_t)S.cap;
    cudaError_t e1 = cudaMalloc(&S.buf, bytes), e2 = cudaMalloc(&S.alt, bytes);
    cudaError_t e3 = cudaMalloc(&S.keys, sizeof(int32_t) * S.cap);
    cudaError_t e4 = cudaMalloc(&S.cell_start, sizeof(int32_t) * (c->nkeys + 1));
    cudaError_t e5 = c->fp64 ? cudaSuccess : cudaMalloc(&S.perm, sizeof(int32_t) * S.cap);
    if (e1 || e2 || e3 || e4 || e5) {
        cudaFree(S.buf); cudaFree(S.alt); cudaFree(S.keys); cudaFree(S.cell_start); cudaFree(S.perm);
        S = Species();
        return fail(c, PP_ENOMEM, "species storage of %zu bytes x 2", bytes);
    }
    S.bind(c->fp64);
    graphs_clear(c);
    *sid = c->nspecies++;
    return PP_OK;
}

extern "C" int pp_set_radiative_cooling(pp_ctx *p, int sid, double coef) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "pp_set_radiative_cooling: NULL context");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (!isfinite(coef) || coef < 0.0) return fail(c, PP_EINVAL, "cooling coefficient must be finite and >= 0");
    c->sp[sid].rad = coef;
    graphs_clear(c);
    return PP_OK;
}

// ---------------------------------------------------------------------------
// Loading
// ---------------------------------------------------------------------------
static int refresh_gauss_reference(Ctx *c) {
    double tmp[16];
    CU(launch_rho(*c, true));
    c->have_G0 = false;
    CU(launch_mesh_diag(*c, tmp));
    CU(cudaStreamSynchronize(c->st));
    c->g0_pending = false;
    return PP_OK;
}

// Loads mark the Gauss reference G_0 as due; it is taken before the next call
// that moves or reads the state, i.e. from the state the loads left (one rho
// deposit however many species and field loads came before).
static int ensure_gauss_reference(Ctx *c) { return c->g0_pending ? refresh_gauss_reference(c) : PP_OK; }

// True when p points to page-locked host memory the device can read directly.
static bool pinned_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

extern "C" int pp_load_particles(pp_ctx *p, int sid, int64_t n, const double *x, const double *y, const double *z,
                                 const double *ux, const double *uy, const double *uz, int on_device) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    Species &S = c->sp[sid];
    if (n < 0) return fail(c, PP_EINVAL, "negative count");
    if (n > 0 && (!x || !y || !z || !ux || !uy || !uz)) return fail(c, PP_EINVAL, "NULL particle array");
    if (S.n + n > S.limit) return fail(c, PP_ENOMEM, "species %d capacity %lld exceeded", sid, (long long)S.limit);
    graphs_clear(c);   // particle counts set launch sizes
    // Device arrays and page-locked host arrays are read in place by the
    // convert kernel (host memory over the host link); pageable host arrays
    // go through a device staging buffer in chunks.
    const double *src[6] = {x, y, z, ux, uy, uz};
    bool direct = on_device != 0;
    if (!direct && n > 0) {
        direct = true;
        for (int k = 0; k < 6; ++k) direct = direct && pinned_host(src[k]);
    }
    const int64_t chunk = direct ? (n > 0 ? n : 1) : ((int64_t)1 << 24);
    double *stage = nullptr;
    if (!direct && n > 0) CU(cudaMalloc(&stage, sizeof(double) * 6 * (size_t)(n < chunk ? n : chunk)));
    int rc = PP_OK;
    cudaError_t e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st);
    if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "particle load: %s", cudaGetErrorString(e));
    for (int64_t off = 0; off < n && rc == PP_OK; off += chunk) {
        int64_t m = n - off < chunk ? n - off : chunk;
        const double *a[6];
        for (int k = 0; k < 6; ++k) {
            if (direct) {
                a[k] = src[k] + off;
            } else {
                double *dst = stage + (size_t)k * (size_t)(n < chunk ? n : chunk);
                e = cudaMemcpyAsync(dst, src[k] + off, sizeof(double) * m, cudaMemcpyHostToDevice, c->st);
                if (e != cudaSuccess) { rc = fail(c, PP_ECUDA, "particle upload: %s", cudaGetErrorString(e)); break; }
                a[k] = dst;
            }
        }
        if (rc != PP_OK) break;
        // converted past the species' count: nothing is appended unless every row is finite
        e = launch_convert_in(*c, sid, S.n + off, m, a[0], a[1], a[2], a[3], a[4], a[5], c->d_status);
        if (e != cudaSuccess) { rc = fail(c, PP_ECUDA, "particle convert: %s", cudaGetErrorString(e)); break; }
    }
    if (rc == PP_OK) {
        e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "particle load: %s", cudaGetErrorString(e));
        else if (*c->h_status & 1) rc = fail(c, PP_ENAN, "non-finite particle value: nothing appended");
        else if (*c->h_status) rc = fail(c, PP_EINVAL, "particle position outside the walls: nothing appended");
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st);
    }
    if (stage) {
        cudaStreamSynchronize(c->st);
        cudaFree(stage);
    }
    if (rc != PP_OK) return rc;
    S.n += n;
    CU(launch_sort(*c, sid));
    if (!c->slab) c->g0_pending = true;   // a slab rank's rho is a share: no reference
    return PP_OK;
}

template <typename R>
__global__ void k_compact_to_padded(Geom g, const double *src, R *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    int i = (int)(t % g.n[0]);
    int64_t r = t / g.n[0];
    int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
    dst[g.at(i, j, k)] = (R)src[t];
}

template <typename R>
__global__ void k_padded_to_compact(Geom g, const R *src, double *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cells()) return;
    int i = (int)(t % g.n[0]);
    int64_t r = t / g.n[0];
    int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
    dst[t] = (double)src[g.at(i, j, k)];
}

static cudaError_t to_padded(Ctx *c, const double *src, void *dst) {
    unsigned b = (unsigned)((c->g.cells() + 255) / 256);
    if (c->fp64) k_compact_to_padded<double><<<b, 256, 0, c->st>>>(c->g, src, (double *)dst);
    else k_compact_to_padded<float><<<b, 256, 0, c->st>>>(c->g, src, (float *)dst);
    ++c->nlaunch;
    return cudaGetLastError();
}

static cudaError_t to_compact(Ctx *c, const void *src, double *dst) {
    unsigned b = (unsigned)((c->g.cells() + 255) / 256);
    if (c->fp64) k_padded_to_compact<double><<<b, 256, 0, c->st>>>(c->g, (const double *)src, dst);
    else k_padded_to_compact<float><<<b, 256, 0, c->st>>>(c->g, (const float *)src, dst);
    ++c->nlaunch;
    return cudaGetLastError();
}

extern "C" int pp_load_fields(pp_ctx *p, const double *const E[3], const double *const B[3], int on_device) {
    Ctx *c = p;
    if (!c || !E || !B) return fail(c, PP_EINVAL, "pp_load_fields: NULL argument");
    for (int a = 0; a < 3; ++a)
        if (!E[a] || !B[a]) return fail(c, PP_EINVAL, "pp_load_fields: NULL component");
    size_t nb = sizeof(double) * (size_t)c->g.cells();
    double *stage = nullptr;
    if (!on_device) CU(cudaMalloc(&stage, nb));
    const double *const *srcs[2] = {E, B};
    void **dsts[2] = {c->E, c->B};
    for (int f = 0; f < 2; ++f)
        for (int a = 0; a < 3; ++a) {
            const double *s = srcs[f][a];
            if (!on_device) {
                CU(cudaMemcpyAsync(stage, s, nb, cudaMemcpyHostToDevice, c->st));
                s = stage;
            }
            CU(to_padded(c, s, dsts[f][a]));
        }
    CU(launch_mirror_fields(*c));   // between walls: the mirror-symmetric part
    CU(launch_ghost_fill(*c, c->E, c->B));
    CU(cudaStreamSynchronize(c->st));
    if (stage) cudaFree(stage);
    c->g0_pending = true;
    return PP_OK;
}

// ---------------------------------------------------------------------------
// Profiling: a pair of events around each phase while enabled.
// ---------------------------------------------------------------------------
static cudaError_t prof_mark(Ctx *c, int phase, bool begin) {
    if (!c->prof) return cudaSuccess;
    if (begin) {
        if (c->prof_n == c->prof_cap) {
            int cap = c->prof_cap ? 2 * c->prof_cap : 256;
            EventPair *nv = (EventPair *)realloc(c->prof_ev, sizeof(EventPair) * cap);
            if (!nv) return cudaErrorMemoryAllocation;
            for (int q = c->prof_cap; q < cap; ++q) {
                nv[q].phase = -1;
                cudaError_t e = cudaEventCreate(&nv[q].a);
                if (e == cudaSuccess) e = cudaEventCreate(&nv[q].b);
                if (e != cudaSuccess) { c->prof_ev = nv; c->prof_cap = q; return e; }
            }
            c->prof_ev = nv;
            c->prof_cap = cap;
        }
        c->prof_ev[c->prof_n].phase = phase;
        return cudaEventRecord(c->prof_ev[c->prof_n].a, c->st);
    }
    cudaError_t e = cudaEventRecord(c->prof_ev[c->prof_n].b, c->st);
    ++c->prof_n;
    return e;
}

// Fold the recorded pairs into the totals (after a synchronisation).
static cudaError_t prof_collect(Ctx *c) {
    for (int q = 0; q < c->prof_n; ++q) {
        float ms = 0.0f;
        cudaError_t e = cudaEventElapsedTime(&ms, c->prof_ev[q].a, c->prof_ev[q].b);
        if (e != cudaSuccess) return e;
        c->prof_ms[c->prof_ev[q].phase] += ms;
    }
    c->prof_n = 0;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// The step
// ---------------------------------------------------------------------------
// The per-step sorted kernel (PP_DEPOSIT_CELLS, and PP_DEPOSIT_AUTO where it
// applies) starts every particle pass from particles sorted by cell (Sec. III:
// the sort between the deposit and the field update of every step).
static bool cells_mode(const Ctx *c) {
    const int m = c->d.deposit_mode;
    return !c->fp64 && (m == PP_DEPOSIT_CELLS || m == PP_DEPOSIT_AUTO) && cells_supported(*c);
}

// The parts of a particle phase around its kernel launch: before it, the
// per-step sort of the per-step sorted kernel when the particles moved, and
// the cleared current; after it, the ghost fold, the images' current between
// walls and the high-order current solve.
static int particle_pre(Ctx *c, bool cells) {
    if (cells) {
        bool stale = false;
        for (int s = 0; s < c->nspecies; ++s) stale = stale || (c->sp[s].n > 0 && !c->sp[s].fresh);
        if (stale) {
            CU(prof_mark(c, PH_SORT, true));
            for (int s = 0; s < c->nspecies; ++s)
                if (!c->sp[s].fresh) CU(launch_sort(*c, s));
            CU(prof_mark(c, PH_SORT, false));
            c->since_sort = 0;
        }
    }
    CU(launch_zero_J(*c));
    CU(cudaMemsetAsync(c->d_nslow, 0, sizeof(unsigned long long), c->st));
    CU(prof_mark(c, PH_PARTICLE, true));
    return PP_OK;
}

static int particle_post(Ctx *c, int only) {
    for (int s = 0; s < c->nspecies; ++s)
        if (only < 0 || s == only) c->sp[s].fresh = false;   // the particles moved
    CU(prof_mark(c, PH_PARTICLE, false));
    CU(prof_mark(c, PH_CURRENT, true));
    CU(launch_fold_J(*c));
    CU(launch_mirror_J(*c));   // between walls: the virtual images' current
    if (c->current_mode == PP_CURRENT_CONSERVING) CU(launch_current_solve(*c));   // eq:jj2 is final
    CU(prof_mark(c, PH_CURRENT, false));
    if (c->prof) ++c->prof_steps;
    if (c->prof && c->prof_n > 4096) {
        CU(cudaStreamSynchronize(c->st));
        CU(prof_collect(c));
    }
    return PP_OK;
}

static int particle_phase(Ctx *c, int only) {
    NvtxRange nvtx("pp particle phase");
    const bool cells = only < 0 && cells_mode(c);
    if (int r = particle_pre(c, cells)) return r;
    bool all_sorted = true;
    for (int s = 0; s < c->nspecies; ++s) all_sorted = all_sorted && (c->sp[s].sorted || c->sp[s].n == 0);
    const int m = c->d.deposit_mode;
    bool tiled = !c->fp64 && !cells && (m == PP_DEPOSIT_TILED || m == PP_DEPOSIT_CELLS ||
                                        (m == PP_DEPOSIT_AUTO && tiled_supported(*c) && all_sorted));
    if (cells) {
        CU(launch_particles_cells(*c));
        if (c->prof) ++c->prof_particle_launches;
    } else if (tiled && only < 0) {
        CU(launch_particles_tiled_all(*c));
        if (c->prof) ++c->prof_particle_launches;
    } else {
        for (int s = 0; s < c->nspecies; ++s) {
            if (only >= 0 && s != only) continue;
            if (c->sp[s].n == 0) continue;
            if (c->fp64) CU(launch_particles_fp64(*c, s));
            else CU(launch_particles_mixed_global(*c, s));
            if (c->prof) ++c->prof_particle_launches;
        }
    }
    return particle_post(c, only);
}

static int field_phase(Ctx *c) {
    NvtxRange nvtx("pp field update");
    CU(prof_mark(c, PH_FIELD, true));
    CU(launch_field_update(*c));
    CU(prof_mark(c, PH_FIELD, false));
    return PP_OK;
}

extern "C" int pp_profile_enable(pp_ctx *p, int enable) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (enable) {
        CU(cudaStreamSynchronize(c->st));
        c->prof_n = 0;
        for (int q = 0; q < PH_N; ++q) c->prof_ms[q] = 0.0;
        c->prof_particle_launches = c->prof_steps = 0;
        c->nlaunch = 0;
    }
    c->prof = enable != 0;
    return PP_OK;
}

extern "C" int pp_profile_read(pp_ctx *p, pp_profile *out) {
    Ctx *c = p;
    if (!c || !out) return fail(c, PP_EINVAL, "pp_profile_read: NULL argument");
    CU(cudaStreamSynchronize(c->st));
    CU(prof_collect(c));
    out->particle_ms = c->prof_ms[PH_PARTICLE];
    out->particle_launches = c->prof_particle_launches;
    out->current_ms = c->prof_ms[PH_CURRENT];
    out->field_ms = c->prof_ms[PH_FIELD];
    out->sort_ms = c->prof_ms[PH_SORT];
    out->steps = c->prof_steps;
    out->kernel_launches = c->nlaunch;
    return PP_OK;
}

extern "C" int pp_sort(pp_ctx *p) {
    NvtxRange nvtx("pp sort");
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    CU(prof_mark(c, PH_SORT, true));
    for (int s = 0; s < c->nspecies; ++s) CU(launch_sort(*c, s));
    CU(prof_mark(c, PH_SORT, false));
    c->since_sort = 0;
    return PP_OK;
}

// The device work of one step: the sort when `sort`, then the particle and
// field phases (four kick-drift substeps for the 4th-order integrator).  Only
// enqueues work; the host state it changes is the J / J' and particle buffer
// swaps, the sorted flags and the last solve's iteration data.
// Open end, injectors or a sliding window: steps change the particle count on
// the host and synchronise at sorts, so they run eagerly.
static bool boundary_dynamic(const Ctx *c) {
    if (!c->wall[0]) return false;
    if (c->open.cells > 0 || c->window.v > 0.0) return true;
    for (int s = 0; s < c->nspecies; ++s)
        if (c->inj[s].ppc > 0.0) return true;
    return false;
}

// Drop the particles that left the box (a sort of each species that may hold
// some; synchronises).
static int compact(Ctx *c) {
    for (int s = 0; s < c->nspecies; ++s)
        if (c->sp[s].may_hold_dead) CU(launch_sort(*c, s));
    return PP_OK;
}

// Drift velocity along x of injector s.
static double inj_vx(const Ctx::Injector &I) {
    return I.u[0] / sqrt(1.0 + I.u[0] * I.u[0] + I.u[1] * I.u[1] + I.u[2] * I.u[2]);
}

// What the open end, the injectors and the window do after a step (Sec. V,
// outflow, injection and sliding window): damp the layer (outgoing particles
// already left in the particle pass), inject the inflow of the step, and shift
// the window when it has moved a cell.
static int boundary_step(Ctx *c) {
    if (c->open.cells > 0 && c->open.mask) {
        CU(launch_damp(*c));
        c->filtered_after_solve = true;   // B moved since the solve: its residual no longer measures it
    }
    const double ny = c->d.ny, nz = c->d.nz;   // the physical box
    for (int s = 0; s < c->nspecies; ++s) {
        const Ctx::Injector &I = c->inj[s];
        if (!(I.ppc > 0.0)) continue;
        const double vx = inj_vx(I);
        const double rate = I.ppc * ny * nz * vx * c->d.dt / c->d.dx;
        const int64_t k = c->step - I.k0;
        const int64_t count = (int64_t)(floor((double)k * rate) - floor((double)(k - 1) * rate));
        Species &S = c->sp[s];
        if (S.n + count > S.limit)
            return fail(c, PP_ENOMEM, "injector of species %d: capacity %lld exceeded", s, (long long)S.limit);
        CU(launch_inject(*c, s, S.n, count, (uint32_t)c->step, 0u, vx * c->d.dt));
        S.n += count;
    }
    if (c->window.v > 0.0) {
        const double f = c->window.v * c->d.dt / c->d.dx;
        const int64_t k = c->step - c->window.k0;
        if (floor((double)k * f) > floor((double)(k - 1) * f)) {
            ++c->window.shifts;
            CU(launch_window_fields(*c));
            c->filtered_after_solve = true;
            for (int s = 0; s < c->nspecies; ++s) {
                CU(launch_window_particles(*c, s));
                c->sp[s].may_hold_dead = true;
            }
            for (int s = 0; s < c->nspecies; ++s) {
                const Ctx::Injector &I = c->inj[s];
                if (!(I.ppc > 0.0)) continue;
                const int64_t count = (int64_t)floor(I.ppc * ny * nz + 0.5);
                Species &S = c->sp[s];
                if (S.n + count > S.limit)
                    return fail(c, PP_ENOMEM, "window layer of species %d: capacity %lld exceeded", s,
                                (long long)S.limit);
                CU(launch_inject(*c, s, S.n, count, (uint32_t)c->window.shifts, 16u, c->d.dx));
                S.n += count;
            }
            if (int r = pp_sort(static_cast<pp_ctx *>(c))) return r;   // cells moved: re-tile
        }
    }
    return PP_OK;
}

static int step_body(Ctx *c, bool sort, bool filter) {
    if (sort) {
        int r = pp_sort(static_cast<pp_ctx *>(c));
        if (r) return r;
    }
    int r = PP_OK;
    // the open end takes outgoing particles at the end of a full step
    const double esc = (c->wall[0] && c->open.cells > 0) ? c->open.escape : 0.0;
    if (esc > 0.0)
        for (int s = 0; s < c->nspecies; ++s) c->sp[s].may_hold_dead = true;
    if (c->order == 4) {
        double a[4], b[4];
        step4_fractions(a, b);
        for (int i = 0; i < 4 && r == PP_OK; ++i) {
            c->kick_dt = b[i] * c->d.dt;
            c->drift_dt = a[i] * c->d.dt;
            c->cheb_sel = (i == 0 || i == 3) ? 1 : 2;
            c->escape_now = i == 3 ? esc : 0.0;
            r = particle_phase(c, -1);
            if (r == PP_OK) r = field_phase(c);
        }
        c->kick_dt = c->drift_dt = c->d.dt;
        c->cheb_sel = 0;
    } else {
        c->escape_now = esc;
        r = particle_phase(c, -1);
        if (r == PP_OK) r = field_phase(c);
    }
    c->escape_now = 0.0;
    if (r == PP_OK && filter) {
        NvtxRange nvtx("pp divergence filter");
        CU(launch_divergence_filter(*c));
    }
    return r;
}

static bool graph_matches(const Ctx *c, const StepGraph &G, bool sort, bool filter) {
    if (!G.valid || G.sort != sort || G.filter != filter || G.J0 != c->J[0]) return false;
    // freshness, a pending permutation and valid keys change what a step
    // launches only for the per-step sorted kernel (elsewhere they stay false)
    const bool cells = cells_mode(c);
    for (int s = 0; s < c->nspecies; ++s) {
        if (G.buf[s] != c->sp[s].buf || G.sorted[s] != c->sp[s].sorted) return false;
        if (cells && (G.fresh[s] != c->sp[s].fresh || G.pending[s] != c->sp[s].perm_pending ||
                      G.keys_valid[s] != c->sp[s].keys_valid))
            return false;
    }
    return true;
}

// Host state a step leaves behind, taken after a capture and re-applied after
// each replay of that capture.
static void graph_save_after(const Ctx *c, StepGraph &G) {
    for (int a = 0; a < 3; ++a) {
        G.J_after[a] = c->J[a];
        G.Jt_after[a] = c->Jt[a];
    }
    for (int s = 0; s < c->nspecies; ++s) {
        G.buf_after[s] = c->sp[s].buf;
        G.alt_after[s] = c->sp[s].alt;
        G.sorted_after[s] = c->sp[s].sorted;
        G.fresh_after[s] = c->sp[s].fresh;
        G.pending_after[s] = c->sp[s].perm_pending;
        G.keys_valid_after[s] = c->sp[s].keys_valid;
    }
    G.since_sort_after = c->since_sort;
    G.last_iters = c->last_iters;
    G.last_kk = c->last_kk;
    G.filtered_after_solve = c->filtered_after_solve;
}

static void graph_apply_after(Ctx *c, const StepGraph &G) {
    for (int a = 0; a < 3; ++a) {
        c->J[a] = G.J_after[a];
        c->Jt[a] = G.Jt_after[a];
    }
    for (int s = 0; s < c->nspecies; ++s) {
        Species &S = c->sp[s];
        S.buf = G.buf_after[s];
        S.alt = G.alt_after[s];
        S.bind(c->fp64);
        S.sorted = G.sorted_after[s];
        S.fresh = G.fresh_after[s];
        S.perm_pending = G.pending_after[s];
        S.keys_valid = G.keys_valid_after[s];
        if (S.sorted) S.nsorted = S.n;   // graph steps neither add nor drop particles
    }
    c->last_iters = G.last_iters;
    c->last_kk = G.last_kk;
    c->filtered_after_solve = G.filtered_after_solve;
    c->since_sort = G.since_sort_after;
}

// One step through the graph cache: replay the capture that starts from the
// current state, or capture it (and launch the capture).  A capture that fails
// leaves the host state as it was and the step runs eagerly.
static int step_graph(Ctx *c, bool sort, bool filter) {
    for (int q = 0; q < kGraphSlots; ++q) {
        StepGraph &G = c->graphs[q];
        if (!graph_matches(c, G, sort, filter)) continue;
        CU(cudaGraphLaunch(G.exec, c->st));
        graph_apply_after(c, G);
        c->nlaunch += G.launches;
        ++c->graph_replays;
        return PP_OK;
    }
    int q = -1;
    for (int k = 0; k < kGraphSlots; ++k)
        if (!c->graphs[k].valid) { q = k; break; }
    if (q < 0) {
        q = c->graph_next;
        c->graph_next = (c->graph_next + 1) % kGraphSlots;
    }
    StepGraph &G = c->graphs[q];
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G = StepGraph();
    G.sort = sort;
    G.filter = filter;
    G.J0 = c->J[0];
    for (int s = 0; s < c->nspecies; ++s) {
        G.buf[s] = c->sp[s].buf;
        G.sorted[s] = c->sp[s].sorted;
        G.fresh[s] = c->sp[s].fresh;
        G.pending[s] = c->sp[s].perm_pending;
        G.keys_valid[s] = c->sp[s].keys_valid;
    }
    // host state before, for a failed capture
    StepGraph before;
    graph_save_after(c, before);
    bool sorted0[PP_MAX_SPECIES], fresh0[PP_MAX_SPECIES], pending0[PP_MAX_SPECIES], keys0[PP_MAX_SPECIES];
    for (int s = 0; s < c->nspecies; ++s) {
        sorted0[s] = c->sp[s].sorted;
        fresh0[s] = c->sp[s].fresh;
        pending0[s] = c->sp[s].perm_pending;
        keys0[s] = c->sp[s].keys_valid;
    }
    int since0 = c->since_sort;
    int64_t nl0 = c->nlaunch;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed);
    int r = e == cudaSuccess ? step_body(c, sort, filter) : PP_ECUDA;
    if (e == cudaSuccess) e = cudaStreamEndCapture(c->st, &graph);
    cudaGraphExec_t exec = nullptr;
    if (r == PP_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (r != PP_OK || e != cudaSuccess || !exec) {
        cudaGetLastError();   // clear a capture error
        if (exec) cudaGraphExecDestroy(exec);
        graph_apply_after(c, before);   // undo the pointer swaps of the capture
        for (int s = 0; s < c->nspecies; ++s) {
            c->sp[s].sorted = sorted0[s];
            c->sp[s].fresh = fresh0[s];
            c->sp[s].perm_pending = pending0[s];
            c->sp[s].keys_valid = keys0[s];
        }
        c->since_sort = since0;
        c->nlaunch = nl0;
        G = StepGraph();
        c->use_graphs = false;   // do not try again on this context
        return step_body(c, sort, filter);
    }
    G.exec = exec;
    G.launches = (int)(c->nlaunch - nl0);
    graph_save_after(c, G);
    G.valid = true;
    ++c->graph_captures;
    CU(cudaGraphLaunch(exec, c->st));
    return PP_OK;
}

extern "C" int pp_step(pp_ctx *p, int nsteps) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (nsteps < 0) return fail(c, PP_EINVAL, "negative step count");
    if (int r = ensure_gauss_reference(c)) return r;
    for (int it = 0; it < nsteps; ++it) {
        bool sort = c->d.sort_interval > 0 && c->since_sort >= c->d.sort_interval;
        bool filter = c->filter_passes > 0 && (c->step + 1) % c->filter_interval == 0;
        const bool dyn = boundary_dynamic(c);
        int r = (c->use_graphs && !c->prof && c->st && !dyn) ? step_graph(c, sort, filter) : step_body(c, sort, filter);
        if (r) return r;
        ++c->step;
        ++c->since_sort;
        if (dyn && (r = boundary_step(c)) != PP_OK) return r;
    }
    return PP_OK;
}

// ---------------------------------------------------------------------------
// Batched form: a step split around a particle kernel launched for many
// contexts at once (pp_batch.cu).  Only contexts that step as one leap-frog
// step through the per-step sorted kernel, with no open end, injector or
// window and no profiling, take this path.
// ---------------------------------------------------------------------------
namespace pp {

bool batch_fusable(const Ctx *c) {
    return cells_mode(c) && c->order == 2 && !boundary_dynamic(c) && !c->prof;
}

int batch_step_pre(Ctx *c) {
    if (int r = ensure_gauss_reference(c)) return r;
    const bool sort = c->d.sort_interval > 0 && c->since_sort >= c->d.sort_interval;
    if (sort) {
        if (int r = pp_sort(static_cast<pp_ctx *>(c))) return r;
    }
    c->kick_dt = c->drift_dt = c->d.dt;
    c->escape_now = 0.0;
    return particle_pre(c, true);
}

int batch_step_post(Ctx *c) {
    int r = particle_post(c, -1);
    if (r == PP_OK) r = field_phase(c);
    if (r == PP_OK && c->filter_passes > 0 && (c->step + 1) % c->filter_interval == 0) {
        CU(launch_divergence_filter(*c));
    }
    if (r == PP_OK) {
        ++c->step;
        ++c->since_sort;
    }
    return r;
}

}  // namespace pp

extern "C" int pp_set_field_solver(pp_ctx *p, int solver) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (solver != PP_FIELD_IMPLICIT && solver != PP_FIELD_EXPLICIT) return fail(c, PP_EINVAL, "unknown field solver");
    if (solver == PP_FIELD_EXPLICIT) {
        // leap-frog stability: dt^2 sum_a Kmax_a^2 < 4
        double h[3] = {c->d.dx, c->d.dy, c->d.dz}, sum = 0.0;
        for (int a = 0; a < 3; ++a) {
            double best = 0.0;
            for (int s = 0; s <= 4000; ++s) {
                double th = M_PI * s / 4000.0;
                double K = 2.0 * (c->fd[0] * sin(0.5 * th) + c->fd[1] * sin(1.5 * th) + c->fd[2] * sin(2.5 * th));
                best = fmax(best, K * K);
            }
            sum += best / (h[a] * h[a]);
        }
        double dt_max = 2.0 / sqrt(sum);
        if (!(c->d.dt < dt_max))
            return fail(c, PP_EINVAL, "the explicit solver needs dt < %.6g on this grid", dt_max);
    }
    c->field_solver = solver;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_current_deposit(pp_ctx *p, int mode) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (mode != PP_CURRENT_CONSERVING && mode != PP_CURRENT_DIRECT) return fail(c, PP_EINVAL, "unknown current deposit");
    c->current_mode = mode;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_divergence_filter(pp_ctx *p, int passes, int interval) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (passes < 0 || interval < 1) return fail(c, PP_EINVAL, "filter needs passes >= 0 and interval >= 1");
    c->filter_passes = passes;
    c->filter_interval = interval;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_open_boundary(pp_ctx *p, int cells, double damping, double escape, int components) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (!c->wall[0]) return fail(c, PP_EINVAL, "an open end needs boundary_x = PP_BOUNDARY_WALLS");
    if (cells < 0 || cells > c->wall[0]) return fail(c, PP_EINVAL, "layer of %d cells outside [0, nx]", cells);
    if (!(damping >= 0.0 && damping <= 1.0)) return fail(c, PP_EINVAL, "damping must lie in [0, 1]");
    if (!(escape >= 0.0 && escape <= (double)c->wall[0])) return fail(c, PP_EINVAL, "escape must lie in [0, nx]");
    if (components < 0 || components > 63) return fail(c, PP_EINVAL, "components is a 6-bit mask");
    c->open.cells = cells;
    c->open.damping = damping;
    c->open.escape = escape;
    c->open.mask = components;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_injector(pp_ctx *p, int sid, double ppc, const double u[3], double u_th, uint64_t seed) {
    Ctx *c = p;
    if (!c || !u) return fail(c, PP_EINVAL, "pp_set_injector: NULL argument");
    if (!c->wall[0]) return fail(c, PP_EINVAL, "an injector needs boundary_x = PP_BOUNDARY_WALLS");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (!(ppc >= 0.0 && ppc < 1e6) || !(u_th >= 0.0 && u_th < 1e6) || !isfinite(u[0]) || !isfinite(u[1]) ||
        !isfinite(u[2]))
        return fail(c, PP_EINVAL, "injector needs 0 <= ppc, 0 <= u_th and a finite drift");
    if (ppc > 0.0 && !(u[0] > 0.0)) return fail(c, PP_EINVAL, "the inflow must move into the box (u_x > 0)");
    Ctx::Injector &I = c->inj[sid];
    I.ppc = ppc;
    for (int a = 0; a < 3; ++a) I.u[a] = u[a];
    I.u_th = u_th;
    I.seed = seed;
    I.k0 = c->step;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_sliding_window(pp_ctx *p, double v) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (!c->wall[0]) return fail(c, PP_EINVAL, "a sliding window needs boundary_x = PP_BOUNDARY_WALLS");
    if (!(v >= 0.0 && v < 1.0)) return fail(c, PP_EINVAL, "window speed must lie in [0, c)");
    c->window.v = v;
    c->window.k0 = c->step;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_set_graphs(pp_ctx *p, int enable) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (enable && !c->st) return fail(c, PP_EINVAL, "step graphs need a context stream other than the legacy default");
    if (int r = compact(c)) return r;   // a capture holds no synchronisation
    c->use_graphs = enable != 0;
    if (!enable) graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_get_graph_stats(pp_ctx *p, int64_t *captures, int64_t *replays) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (captures) *captures = c->graph_captures;
    if (replays) *replays = c->graph_replays;
    return PP_OK;
}

extern "C" int pp_set_integrator(pp_ctx *p, int order) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (order != 2 && order != 4) return fail(c, PP_EINVAL, "integrator order must be 2 or 4");
    c->order = order;
    graphs_clear(c);
    return PP_OK;
}

extern "C" int pp_deposit(pp_ctx *p, int sid) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (sid < -1 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (int r0 = ensure_gauss_reference(c)) return r0;
    int r = particle_phase(c, sid);
    if (r == PP_OK) ++c->since_sort;
    return r;
}

extern "C" int pp_field_update(pp_ctx *p) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (int r = ensure_gauss_reference(c)) return r;
    return field_phase(c);
}

extern "C" int pp_set_tuning(pp_ctx *p, int sort_interval, int deposit_mode) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (sort_interval < 0) return fail(c, PP_EINVAL, "sort_interval must be >= 0");
    if (deposit_mode < 0 || deposit_mode > 3) return fail(c, PP_EINVAL, "unknown deposit_mode");
    if ((deposit_mode == PP_DEPOSIT_TILED || deposit_mode == PP_DEPOSIT_CELLS) && !tiled_supported(*c))
        return fail(c, PP_EINVAL, "the tiled deposits need PP_MIXED32 and grid sizes that are multiples of 8");
    c->d.sort_interval = sort_interval;
    c->d.deposit_mode = deposit_mode;
    graphs_clear(c);
    return PP_OK;
}

static int status_code(int bits) {
    if (bits & ST_BOUNDS) return PP_EBOUNDS;
    if (bits & ST_TIMEOUT) return PP_ETIMEOUT;
    if (bits & ST_NAN) return PP_ENAN;
    if (bits & ST_CFL) return PP_ECFL;
    if (bits & ST_NOCONV) return PP_ENOCONV;
    if (bits & ST_RANGE) return PP_EINVAL;
    return PP_OK;
}

extern "C" int pp_sync(pp_ctx *p) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    CU(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    CU(cudaStreamSynchronize(c->st));
    int code = status_code(*c->h_status);
    if (code) return fail(c, code, "device status 0x%x (NaN=1, CFL=2, relaxation=4, range=8, bounds=16, timeout=32)", *c->h_status);
    return PP_OK;
}

extern "C" int pp_diagnostics(pp_ctx *p, pp_diag *out) {
    Ctx *c = p;
    if (!c || !out) return fail(c, PP_EINVAL, "pp_diagnostics: NULL argument");
    if (int r = ensure_gauss_reference(c)) return r;
    if (int r = compact(c)) return r;
    int st = pp_sync(p);
    memset(out, 0, sizeof(*out));
    out->status = st;
    double mesh[16], kin[PP_MAX_SPECIES];
    unsigned long long nslow = 0;
    CU(cudaMemcpyAsync(&nslow, c->d_nslow, sizeof nslow, cudaMemcpyDeviceToHost, c->st));
    CU(launch_rho(*c, true));
    CU(launch_kinetic(*c, c->d_out + 16));
    CU(launch_mesh_diag(*c, mesh));
    CU(cudaMemcpyAsync(kin, c->d_out + 16, sizeof(double) * PP_MAX_SPECIES, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    double dV = c->d.dx * c->d.dy * c->d.dz;
    // between walls: the physical part of the extended mesh (half per walled axis)
    const double box = (c->wall[0] ? 0.5 : 1.0) * (c->wall[1] ? 0.5 : 1.0) * (c->wall[2] ? 0.5 : 1.0);
    out->step = c->step;
    out->time = c->step * c->d.dt;
    out->energy_E = mesh[0] * dV * box;
    out->energy_B = mesh[1] * dV * box;
    out->energy_Ex = mesh[2] * dV * box;
    out->charge = mesh[3] * dV * box;
    out->rho_max = mesh[4];
    out->gauss_max = mesh[5];
    out->gauss_drift_max = mesh[6];
    out->divB_max = mesh[7];
    out->relax_residual = (c->last_iters > 0 && mesh[9] > 0.0) ? mesh[8] / mesh[9] : 0.0;
    out->relax_iters = c->last_iters;
    for (int s = 0; s < c->nspecies; ++s) {
        out->kinetic[s] = kin[s];
        out->kinetic_total += kin[s];
        out->n_particles += c->sp[s].n;
    }
    out->n_slow = (int64_t)nslow;
    // a divergence filter moves B after the solve: the residual then includes
    // the filter's correction and is reported but not checked
    if (c->last_iters > 0 && !c->filtered_after_solve && out->relax_residual > 10.0 * c->d.relax_tol &&
        out->status == PP_OK)
        out->status = PP_ENOCONV;
    return PP_OK;
}

extern "C" int pp_get_fields(pp_ctx *p, double *const E[3], double *const B[3], double *const J[3]) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    size_t nb = sizeof(double) * (size_t)c->g.cells();
    double *stage = nullptr;
    CU(cudaMalloc(&stage, nb));
    double *const *dsts[3] = {E, B, J};
    void **srcs[3] = {c->E, c->B, c->J};
    int rc = PP_OK;
    for (int f = 0; f < 3 && rc == PP_OK; ++f) {
        if (!dsts[f]) continue;
        for (int a = 0; a < 3; ++a) {
            if (!dsts[f][a]) continue;
            cudaError_t e = to_compact(c, srcs[f][a], stage);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dsts[f][a], stage, nb, cudaMemcpyDeviceToHost, c->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
            if (e != cudaSuccess) { rc = fail(c, PP_ECUDA, "field readback: %s", cudaGetErrorString(e)); break; }
        }
    }
    cudaFree(stage);
    return rc;
}

extern "C" int pp_check_bounded_wait(pp_ctx *p, int deliver, long long limit_ns) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (limit_ns < 1 || limit_ns > 10000000000ll) return fail(c, PP_EINVAL, "limit_ns %lld outside 1 .. 1e10", limit_ns);
    int rc = pp_sync(p);   // earlier work's status first
    if (rc != PP_OK) return rc;
    CU(launch_wait_check(c->st, c->d_status, deliver, (uint64_t)limit_ns));
    return pp_sync(p);
}

// ---------------------------------------------------------------------------
// z-slab decomposition (multi-GPU): the current of one rank's particles out
// and the summed current in, and the particles that left the rank's slab.
// ---------------------------------------------------------------------------
extern "C" int pp_get_current(pp_ctx *p, double *const J[3], int on_device) {
    Ctx *c = p;
    if (!c || !J || !J[0] || !J[1] || !J[2]) return fail(c, PP_EINVAL, "pp_get_current: NULL argument");
    const size_t nb = sizeof(double) * (size_t)c->g.cells();
    if (on_device) {
        for (int a = 0; a < 3; ++a) CU(to_compact(c, c->J[a], J[a]));
        return PP_OK;
    }
    double *stage = nullptr;
    CU(cudaMalloc(&stage, nb));
    int rc = PP_OK;
    for (int a = 0; a < 3 && rc == PP_OK; ++a) {
        cudaError_t e = to_compact(c, c->J[a], stage);
        if (e == cudaSuccess) e = cudaMemcpyAsync(J[a], stage, nb, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "current readback: %s", cudaGetErrorString(e));
    }
    cudaFree(stage);
    return rc;
}

extern "C" int pp_set_current(pp_ctx *p, const double *const J[3], int on_device) {
    Ctx *c = p;
    if (!c || !J || !J[0] || !J[1] || !J[2]) return fail(c, PP_EINVAL, "pp_set_current: NULL argument");
    graphs_clear(c);
    const size_t nb = sizeof(double) * (size_t)c->g.cells();
    if (on_device) {
        for (int a = 0; a < 3; ++a) CU(to_padded(c, J[a], c->J[a]));
        return PP_OK;
    }
    double *stage = nullptr;
    CU(cudaMalloc(&stage, nb));
    int rc = PP_OK;
    for (int a = 0; a < 3 && rc == PP_OK; ++a) {
        cudaError_t e = cudaMemcpyAsync(stage, J[a], nb, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = to_padded(c, stage, c->J[a]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "current upload: %s", cudaGetErrorString(e));
    }
    cudaFree(stage);
    return rc;
}

extern "C" int pp_set_slab(pp_ctx *p, double z_lo, double z_hi) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (c->wall[2]) return fail(c, PP_EINVAL, "pp_set_slab: z must be periodic");
    const double Lz = c->g.n[2] * c->d.dz;
    if (!(z_lo >= 0.0 && z_lo < z_hi && z_hi <= Lz)) return fail(c, PP_EINVAL, "pp_set_slab: need 0 <= z_lo < z_hi <= Lz");
    c->slab = true;
    c->slab_lo = z_lo;
    c->slab_hi = z_hi;
    return PP_OK;
}

extern "C" int pp_extract_particles(pp_ctx *p, int sid, int64_t cap, double *x, double *y, double *z, double *ux,
                                    double *uy, double *uz, int on_device, int64_t *n_out) {
    Ctx *c = p;
    if (!c || !n_out || cap < 0) return fail(c, PP_EINVAL, "pp_extract_particles: bad argument");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (!c->slab) return fail(c, PP_EINVAL, "pp_extract_particles: no slab set (pp_set_slab)");
    const double z_lo = c->slab_lo, z_hi = c->slab_hi;
    double *const dst[6] = {x, y, z, ux, uy, uz};
    for (int k = 0; k < 6 && cap > 0; ++k)
        if (!dst[k]) return fail(c, PP_EINVAL, "pp_extract_particles: NULL output array");
    Species &S = c->sp[sid];
    *n_out = 0;
    if (S.n == 0) return PP_OK;
    graphs_clear(c);
    unsigned long long *d_count = nullptr;
    CU(cudaMalloc(&d_count, sizeof(unsigned long long)));
    double *stage = nullptr;
    int rc = PP_OK;
    unsigned long long h_count = 0;
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), c->st);
    if (e == cudaSuccess) e = launch_extract(*c, sid, z_lo, z_hi, 0, 0, d_count, dst);   // count first
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_count, d_count, sizeof h_count, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "particle extraction: %s", cudaGetErrorString(e));
    if (rc == PP_OK && (int64_t)h_count > cap)
        rc = fail(c, PP_ENOMEM, "pp_extract_particles: %lld particles left the slab, room for %lld",
                  (long long)h_count, (long long)cap);
    if (rc == PP_OK && h_count > 0) {
        double *out[6];
        if (on_device) {
            for (int k = 0; k < 6; ++k) out[k] = dst[k];
        } else if ((e = cudaMalloc(&stage, 6 * sizeof(double) * h_count)) == cudaSuccess) {
            for (int k = 0; k < 6; ++k) out[k] = stage + (size_t)k * h_count;
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), c->st);
        if (e == cudaSuccess) e = launch_extract(*c, sid, z_lo, z_hi, 1, (int64_t)h_count, d_count, out);
        for (int k = 0; k < 6 && e == cudaSuccess && !on_device; ++k)
            e = cudaMemcpyAsync(dst[k], out[k], sizeof(double) * h_count, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "particle extraction: %s", cudaGetErrorString(e));
        if (rc == PP_OK) {   // drop them now: the compacting sort reads back the new count
            S.may_hold_dead = true;
            if ((e = launch_sort(*c, sid)) != cudaSuccess) rc = fail(c, PP_ECUDA, "compaction: %s", cudaGetErrorString(e));
        }
    }
    cudaFree(stage);
    cudaFree(d_count);
    if (rc == PP_OK) *n_out = (int64_t)h_count;
    return rc;
}

extern "C" int pp_get_rho(pp_ctx *p, double *rho) {
    Ctx *c = p;
    if (!c || !rho) return fail(c, PP_EINVAL, "pp_get_rho: NULL argument");
    CU(launch_rho(*c, true));
    CU(cudaMemcpyAsync(rho, c->rho, sizeof(double) * c->g.cells(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return PP_OK;
}

extern "C" int pp_get_grid(pp_ctx *p, pp_grid_desc *desc, int *nspecies) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (desc) *desc = c->d;
    if (nspecies) *nspecies = c->nspecies;
    return PP_OK;
}

extern "C" int pp_get_count(pp_ctx *p, int sid, int64_t *n) {
    Ctx *c = p;
    if (!c || !n) return fail(c, PP_EINVAL, "pp_get_count: NULL argument");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (int r = compact(c)) return r;
    *n = c->sp[sid].n;
    return PP_OK;
}

extern "C" int pp_get_particles(pp_ctx *p, int sid, double *x, double *y, double *z, double *ux, double *uy,
                                double *uz) {
    Ctx *c = p;
    if (!c) return fail(c, PP_EINVAL, "NULL context");
    if (sid < 0 || sid >= c->nspecies) return fail(c, PP_EINVAL, "no species %d", sid);
    if (int r = compact(c)) return r;
    Species &S = c->sp[sid];
    if (S.n == 0) return PP_OK;
    if (!x || !y || !z || !ux || !uy || !uz) return fail(c, PP_EINVAL, "NULL particle array");
    double *stage = nullptr;
    size_t nb = sizeof(double) * (size_t)S.n;
    CU(cudaMalloc(&stage, nb * 6));
    double *d[6];
    for (int k = 0; k < 6; ++k) d[k] = stage + (size_t)k * S.n;
    double *h[6] = {x, y, z, ux, uy, uz};
    int rc = PP_OK;
    cudaError_t e = launch_convert_out(*c, sid, d[0], d[1], d[2], d[3], d[4], d[5]);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaMemcpyAsync(h[k], d[k], nb, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) rc = fail(c, PP_ECUDA, "particle readback: %s", cudaGetErrorString(e));
    cudaFree(stage);
    return rc;
}

// ---------------------------------------------------------------------------
// Checkpoint / restart (FP64 blocks, independent of the precision form)
// ---------------------------------------------------------------------------
// Format 2 adds each species' radiative-cooling coefficient, format 3 the
// integrator order, format 4 the field solver, format 5 the current deposit
// and the divergence filter; older files restore with the defaults.
static const char kMagic[8] = {'P', 'P', 'G', 'B', '3', '0', '0', '8'};

extern "C" int pp_save(pp_ctx *p, const char *path) {
    Ctx *c = p;
    if (!c || !path) return fail(c, PP_EINVAL, "pp_save: NULL argument");
    if (int r = compact(c)) return r;   // counts written below must be final
    FILE *f = fopen(path, "wb");
    if (!f) return fail(c, PP_EINVAL, "cannot open %s for writing", path);
    int64_t N = c->g.cells();
    std::vector<double> buf((size_t)N * 6);
    double *E[3] = {buf.data(), buf.data() + N, buf.data() + 2 * N};
    double *B[3] = {buf.data() + 3 * N, buf.data() + 4 * N, buf.data() + 5 * N};
    int rc = pp_get_fields(p, E, B, nullptr);
    pp_grid_desc d = c->d;
    d.stream = nullptr;
    bool ok = rc == PP_OK;
    ok = ok && fwrite(kMagic, 1, 8, f) == 8 && fwrite(&d, sizeof d, 1, f) == 1;
    ok = ok && fwrite(&c->step, sizeof c->step, 1, f) == 1 && fwrite(&c->nspecies, sizeof(int), 1, f) == 1 &&
         fwrite(&c->order, sizeof(int), 1, f) == 1 && fwrite(&c->field_solver, sizeof(int), 1, f) == 1 &&
         fwrite(&c->current_mode, sizeof(int), 1, f) == 1 && fwrite(&c->filter_passes, sizeof(int), 1, f) == 1 &&
         fwrite(&c->filter_interval, sizeof(int), 1, f) == 1;
    ok = ok && fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
    for (int s = 0; s < c->nspecies && ok; ++s) {
        Species &S = c->sp[s];
        pp_species_desc sd{S.q, S.m, S.w, S.limit};
        ok = fwrite(&sd, sizeof sd, 1, f) == 1 && fwrite(&S.n, sizeof S.n, 1, f) == 1 &&
             fwrite(&S.rad, sizeof S.rad, 1, f) == 1;
        std::vector<double> pb((size_t)S.n * 6);
        if (ok && S.n) {
            rc = pp_get_particles(p, s, pb.data(), pb.data() + S.n, pb.data() + 2 * S.n, pb.data() + 3 * S.n,
                                  pb.data() + 4 * S.n, pb.data() + 5 * S.n);
            ok = rc == PP_OK && fwrite(pb.data(), sizeof(double), pb.size(), f) == pb.size();
        }
    }
    // format 7: open end, window and injectors
    ok = ok && fwrite(&c->open, sizeof c->open, 1, f) == 1 && fwrite(&c->window, sizeof c->window, 1, f) == 1;
    for (int s = 0; s < c->nspecies && ok; ++s) ok = fwrite(&c->inj[s], sizeof c->inj[s], 1, f) == 1;
    if (fclose(f) != 0) ok = false;
    if (!ok) return rc != PP_OK ? rc : fail(c, PP_EINVAL, "write to %s failed", path);
    return PP_OK;
}

extern "C" int pp_restore(pp_ctx **out, const char *path, void *stream) {
    Ctx *c = nullptr;
    if (!out || !path) return fail(c, PP_EINVAL, "pp_restore: NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(c, PP_EINVAL, "cannot open %s", path);
    char magic[8];
    pp_grid_desc d;
    int64_t step = 0;
    int ns = 0;
    int order = 2, solver = PP_FIELD_IMPLICIT, cmode = PP_CURRENT_CONSERVING, fpasses = 0, finterval = 1;
    // formats 1-5 wrote the descriptor up to boundary_x, formats 6-7 up to boundary_y
    memset(&d, 0, sizeof d);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 7) == 0 && magic[7] >= '1' && magic[7] <= '8' &&
              fread(&d, magic[7] >= '8' ? sizeof d
                                        : (magic[7] >= '6' ? offsetof(pp_grid_desc, boundary_y)
                                                           : offsetof(pp_grid_desc, boundary_x)),
                    1, f) == 1 &&
              fread(&step, sizeof step, 1, f) == 1 && fread(&ns, sizeof ns, 1, f) == 1 && ns >= 0 &&
              ns <= PP_MAX_SPECIES && (magic[7] < '3' || fread(&order, sizeof order, 1, f) == 1) &&
              (magic[7] < '4' || fread(&solver, sizeof solver, 1, f) == 1) &&
              (magic[7] < '5' || (fread(&cmode, sizeof cmode, 1, f) == 1 && fread(&fpasses, sizeof fpasses, 1, f) == 1 &&
                                  fread(&finterval, sizeof finterval, 1, f) == 1));
    if (!ok) { fclose(f); return fail(c, PP_EINVAL, "%s is not a checkpoint of this library", path); }
    d.stream = stream;
    pp_ctx *p = nullptr;
    int rc = pp_init_grid(&p, &d);
    if (rc != PP_OK && rc != PP_WSTAB) { fclose(f); return rc; }
    c = p;
    rc = pp_set_integrator(p, order);
    if (rc == PP_OK) rc = pp_set_field_solver(p, solver);
    if (rc == PP_OK) rc = pp_set_current_deposit(p, cmode);
    if (rc == PP_OK) rc = pp_set_divergence_filter(p, fpasses, finterval);
    int64_t N = c->g.cells();
    std::vector<double> buf((size_t)N * 6);
    ok = rc == PP_OK && fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
    const double *E[3] = {buf.data(), buf.data() + N, buf.data() + 2 * N};
    const double *B[3] = {buf.data() + 3 * N, buf.data() + 4 * N, buf.data() + 5 * N};
    if (ok) rc = pp_load_fields(p, E, B, 0);
    for (int s = 0; s < ns && ok && rc == PP_OK; ++s) {
        pp_species_desc sd;
        int64_t n = 0;
        int sid = -1;
        double rad = 0.0;
        ok = fread(&sd, sizeof sd, 1, f) == 1 && fread(&n, sizeof n, 1, f) == 1 && n >= 0 && n <= sd.capacity &&
             (magic[7] < '2' || fread(&rad, sizeof rad, 1, f) == 1);
        if (!ok) break;
        rc = pp_init_species(p, &sd, &sid);
        if (rc == PP_OK) rc = pp_set_radiative_cooling(p, sid, rad);
        std::vector<double> pb((size_t)n * 6);
        if (rc == PP_OK) ok = fread(pb.data(), sizeof(double), pb.size(), f) == pb.size();
        if (rc == PP_OK && ok && n)
            rc = pp_load_particles(p, sid, n, pb.data(), pb.data() + n, pb.data() + 2 * n, pb.data() + 3 * n,
                                   pb.data() + 4 * n, pb.data() + 5 * n, 0);
    }
    if (ok && rc == PP_OK && magic[7] >= '7') {
        Ctx::OpenEnd open;
        Ctx::Window window;
        ok = fread(&open, sizeof open, 1, f) == 1 && fread(&window, sizeof window, 1, f) == 1;
        if (ok && c->wall[0]) {   // validated through the setters, then the run's state taken over
            rc = pp_set_open_boundary(p, open.cells, open.damping, open.escape, open.mask);
            if (rc == PP_OK) rc = pp_set_sliding_window(p, window.v);
            c->window = window;
        }
        for (int s = 0; s < ns && ok && rc == PP_OK; ++s) {
            Ctx::Injector I;
            ok = fread(&I, sizeof I, 1, f) == 1;
            if (ok && c->wall[0]) {
                rc = pp_set_injector(p, s, I.ppc, I.u, I.u_th, I.seed);
                c->inj[s] = I;
            }
        }
    }
    fclose(f);
    if (!ok || rc != PP_OK) {
        int code = rc != PP_OK ? rc : PP_EINVAL;
        snprintf(g_last_error, sizeof g_last_error, "restore of %.200s failed: %.280s", path, c->err[0] ? c->err : "truncated file");
        pp_destroy(p);
        return code;
    }
    c->step = step;
    *out = p;
    return PP_OK;
}
