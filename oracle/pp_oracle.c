/*
 * pp_oracle.c -- plain, slow, FP64 CPU oracle of the Photon-Plasma particle step
 * (Haugboelle, Frederiksen & Nordlund, "Photon-Plasma: a modern high-order
 * particle-in-cell code", arXiv:1211.4575).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Every loop here is a literal transcription of a definition in the paper (cited
 * per function by section / equation label); there is no blocking, tiling,
 * sorting or fusion.  Periodic boundaries use modular indexing.
 *
 * Conventions (the paper leaves the normalisation free; this oracle fixes it):
 *   c = eps0 = mu0 = 1.
 *   Positions are physical, x in [0, n*dx).  Mesh index i stands for x = i*dx.
 *   Yee staggering (Sec. III, Fig. "Spatial staggering"): rho at (i,j,k);
 *   E_x, J_x at (i+1/2, j, k); B_x at (i, j+1/2, k+1/2); cyclic for y, z.
 *   A component at a half-integer position along an axis is stored at the index
 *   of the node just below it.
 *   Arrays are x-fastest: a[i + n0*(j + n1*k)].
 *
 * Readings of the paper that this oracle takes (where it is silent or garbled):
 *   R1  6th-order coefficient a = 75/64, not the printed 25/21: only 75/64
 *       satisfies the Taylor conditions with the printed b = -25/384,
 *       c = 3/640 (a + 3b + 5c = 1, a + 27b + 125c = 0, a + 243b + 3125c = 0).
 *       4th order: a = 9/8, b = -1/24.  2nd order: a = 1.
 *   R2  The directional charge change obeys d^-_i J_i = -D rho_i (eq:cc1 fixes
 *       the sign; eq:jj3 as printed drops it).
 *   R3  The current term of eq:EllipticB enters with a plus sign: substituting
 *       eq:enplus1 into eq:bnplus1 gives + alpha c^2 mu0 dt^2 curl^+ J.
 *   R4  Periodic current: the per-line integration constant left by the prefix
 *       sum of Sec. III "Charge conserving current density" is fixed by the
 *       line mean of each particle's compact (2nd-order) current, i.e. by the
 *       first moment of its D rho along the line.
 *   R5  The unspecified successive relaxation of eq:EllipticB is read as Jacobi iteration.
 *   R6  Each field component is gathered from its own staggered nodes with the
 *       same weight function as the deposit (eq:pfields, eq:rho2).
 *   R16 Radiative cooling (Sec. "Radiative cooling") is the explicit form the
 *       paper settles on: no iteration, so the proper acceleration inside the
 *       radiated power of eq:prad is the Lorentz one, (p+^EM - p-)/dt, and
 *       p0 = (p+^EM + p-)/2.  The coefficient mu0 q^2/(6 pi m c) is a species
 *       parameter: in a normalised code it depends on the physical unit of
 *       length, which the paper fixes elsewhere.  A particle with p0 = 0 does
 *       not radiate (eq:udot has no direction there).
 *   R17 The 4th-order symplectic step (Sec. III, the passage on the symmetric
 *       fourth-order integrator of Yoshida / Forest & Ruth / Candy & Rozmus)
 *       is four leap-frog substeps, each a kick of b_i dt followed by a drift
 *       of a_i dt, with b = (0, w1, w0, w1), a = (w1/2, (w0+w1)/2, (w0+w1)/2,
 *       w1/2), w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3) w1.  Each kick is then
 *       centred on the position time, the condition the paper states.  The
 *       fields, with positions and charge in the paper's pairing of conjugate
 *       variables, advance in the drifts: the field update of eq:bnplus1 /
 *       eq:enplus1 runs with dt -> a_i dt and the current of that drift.
 *       Positions and proper velocities are both at t at a step boundary.
 *   R18 The explicit 6th-order FDTD solver of the cold-beam comparison (Sec.
 *       VIII, fig:coldbeam) is Yee's leap-frog with the same staggered
 *       differences, B split into two half steps so that E and B stay at the
 *       same time as in the implicit scheme:
 *         B^{n+1/2} = B^n - dt/2 curl^+ E^n,
 *         E^{n+1}   = E^n + dt (curl^- B^{n+1/2} - J),
 *         B^{n+1}   = B^{n+1/2} - dt/2 curl^+ E^{n+1}.
 *   R19 The direct current eq:jj2 (the original code's method, Sec. III after
 *       eq:penta) sums q w v W over particles with each component on its own
 *       staggered nodes (like E), W taken at the middle of the move,
 *       (x^n + x^{n+1})/2, and v = u^{n+1/2}/gamma: J^{n+1/2} without the
 *       high-order current solve, which belongs to the charge-conserving form.
 *   R20 The divergence filter (the Gauss-Seidel filter of E, and the
 *       periodic filter of E and B of long FP32 runs): each pass is one
 *       simultaneous smoothing step E += tau grad^+(div^- E - rho),
 *       B += tau grad^-(div^+ B), tau = 1 / max(sum_a K_a^2), the largest
 *       eigenvalue of -div grad, which removes the Nyquist-scale error in one
 *       pass and damps every other non-constant mode.  Gauss-Seidel ordering
 *       is sequential; the simultaneous form damps the same error.
 *   R21 Reflecting walls (Sec. V "Boundary conditions") are the virtual-image
 *       system in the mirror-extended box (oracle/__init__.py, WallSimulation).
 *   R22 The outflow layer (same section): the paper gives no profile.  Each
 *       step the chosen field components are multiplied by
 *       1 - damping ((cells - d) / cells)^2 at distance d < cells (in cells,
 *       at the component's own staggered position) from the open end.  The
 *       paper's perpendicular components are read as those transverse to the
 *       boundary normal (E_y, E_z, B_y, B_z), the fields of waves leaving along
 *       x; the component set is a parameter.  A particle leaves the box when
 *       a step ends with it moving outward (u_x < 0) closer than `escape`
 *       cells to the open end: until then it deposits like any other.
 *   R23 The injector (Sec. V "Sliding window and injection of particles") is
 *       fed by Philox4x32-10 draws (Salmon et al., SC'11), counter
 *       (index, 0, step, stream), key = the 64-bit seed.  Per step it adds the
 *       inflow that crossed the open end during the step: floor(k r) -
 *       floor((k-1) r) particles at the k-th step since it was set, r = ppc ny
 *       nz v_x dt / dx, v the drift velocity; positions uniform in the slab
 *       [0, v_x dt) x [0, Ly) x [0, Lz), proper velocity = drift + u_th times
 *       three standard normals (Box-Muller).  Positions come from stream 0,
 *       shared by every species, so that species injected with the same seed
 *       and density land on the same points (neutral pairs); velocities from
 *       stream 1 + species.
 *   R24 The sliding window moves the box one cell against x (its content one
 *       cell up) at the k-th step since it was set whenever floor(k v dt / dx)
 *       grows: v (t - t_old) > dx with t_old advanced by dx / v, so that the
 *       window keeps speed v on average.  The top layer and the particles in it
 *       leave, fields of the new bottom layer are zero, and every species with
 *       an injector gets a layer of round(ppc ny nz) particles uniform in
 *       [0, dx) (streams 16 and 17 + species, the shift count as the step).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n[3];            /* cells per axis */
    double d[3];         /* cell size per axis */
    double dt;           /* time step */
    int field_order;     /* 2, 4 or 6 */
    double alpha;        /* de-centering of eq:bnplus1 / eq:enplus1 */
    int shape_order;     /* 0 NGP, 1 CIC, 2 TSC, 3 PCS */
    int pusher;          /* 0 Vay, 1 Boris */
    int relax_max_iter;  /* iteration cap of the relaxation */
    double relax_tol;    /* relative max-norm residual target */
    int field_solver;    /* 0: implicit (eq:EllipticB); 1: explicit FDTD (reading R18) */
    int current_mode;    /* 0: charge-conserving (eq:jj6); 1: direct eq:jj2 (reading R19) */
} orc_grid;

typedef struct {
    double q, m, w;      /* charge, mass, number density per macro-particle */
    int64_t n;           /* number of macro-particles */
    double *x, *y, *z;   /* positions */
    double *ux, *uy, *uz;/* proper velocity gamma*v, staggered to t - dt/2 */
    double rad;          /* mu0 q^2 / (6 pi m c) of eq:udot; 0 = no radiative cooling */
} orc_species;

typedef struct {
    double energy_E, energy_B, energy_Ex;
    double kinetic;
    double charge;
    double gauss_max;    /* max |div^- E - rho| */
    double rho_max;
    double divB_max;     /* max |div^+ B| */
    int relax_iters;
    double relax_residual;
} orc_diag;

/* ------------------------------------------------------------------ */
/* Weight functions W^0..W^3 (Sec. II, list after eq:weightfunction).  */
/* delta = (x_c - x_p)/dx.                                              */
/* ------------------------------------------------------------------ */
double orc_weight(int order, double delta)
{
    double ad = fabs(delta);
    switch (order) {
    case 0: /* NGP */
        return ad <= 0.5 ? 1.0 : 0.0;
    case 1: /* CIC */
        return ad < 1.0 ? 1.0 - ad : 0.0;
    case 2: /* TSC */
        if (ad < 0.5) return 0.75 - delta * delta;
        if (ad < 1.5) return 0.5 * (1.5 - ad) * (1.5 - ad);
        return 0.0;
    case 3: /* PCS */
        if (ad < 1.0) return (4.0 - 6.0 * delta * delta + 3.0 * ad * ad * ad) / 6.0;
        if (ad < 2.0) return (2.0 - ad) * (2.0 - ad) * (2.0 - ad) / 6.0;
        return 0.0;
    }
    return 0.0;
}

/* Staggered difference coefficients (Sec. III "Solving Maxwell's equations"),
 * with reading R1 for the 6th-order a. */
void orc_fd_coeffs(int order, double k[3])
{
    if (order == 6) { k[0] = 75.0 / 64.0; k[1] = -25.0 / 384.0; k[2] = 3.0 / 640.0; }
    else if (order == 4) { k[0] = 9.0 / 8.0; k[1] = -1.0 / 24.0; k[2] = 0.0; }
    else { k[0] = 1.0; k[1] = 0.0; k[2] = 0.0; }
}

static int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static int64_t idx3(const orc_grid *g, int i, int j, int k)
{
    return (int64_t)wrapi(i, g->n[0]) +
           (int64_t)g->n[0] * ((int64_t)wrapi(j, g->n[1]) + (int64_t)g->n[1] * wrapi(k, g->n[2]));
}

static int64_t ncells(const orc_grid *g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }

/* Staggering of the three field families.  stag[a] = 1: the component sits at
 * a half-integer position along axis a. */
static void stag_E(int comp, int s[3]) { s[0] = s[1] = s[2] = 0; s[comp] = 1; }
static void stag_B(int comp, int s[3]) { s[0] = s[1] = s[2] = 1; s[comp] = 0; }

/* ------------------------------------------------------------------ */
/* Staggered first derivatives along one axis (Sec. III, Fig.          */
/* "diffoper").  dir = +1: input on integer nodes, output at i+1/2     */
/* (stored at i).  dir = -1: input at half nodes (i stands for i+1/2), */
/* output on integer node i.                                           */
/* ------------------------------------------------------------------ */
void orc_diff(const orc_grid *g, int order, int axis, int dir, const double *f, double *out)
{
    double kc[3];
    orc_fd_coeffs(order, kc);
    double inv = 1.0 / g->d[axis];
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                int p[3] = {i, j, k};
                double acc = 0.0;
                for (int m = 1; m <= 3; ++m) {
                    int hi[3] = {i, j, k}, lo[3] = {i, j, k};
                    if (dir > 0) { hi[axis] = p[axis] + m;     lo[axis] = p[axis] + 1 - m; }
                    else         { hi[axis] = p[axis] + m - 1; lo[axis] = p[axis] - m; }
                    acc += kc[m - 1] * (f[idx3(g, hi[0], hi[1], hi[2])] - f[idx3(g, lo[0], lo[1], lo[2])]);
                }
                out[idx3(g, i, j, k)] = acc * inv;
            }
}

/* curl with up-shifted derivatives (acts on E-located data, result B-located). */
static void curl_plus(const orc_grid *g, double *const F[3], double *out[3], double *tmp)
{
    int o = g->field_order;
    int64_t N = ncells(g);
    /* out_x = d_y^+ F_z - d_z^+ F_y, and cyclic */
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        orc_diff(g, o, b, +1, F[c], out[a]);
        orc_diff(g, o, c, +1, F[b], tmp);
        for (int64_t q = 0; q < N; ++q) out[a][q] -= tmp[q];
    }
}

/* curl with down-shifted derivatives (acts on B-located data, result E-located). */
static void curl_minus(const orc_grid *g, double *const F[3], double *out[3], double *tmp)
{
    int o = g->field_order;
    int64_t N = ncells(g);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        orc_diff(g, o, b, -1, F[c], out[a]);
        orc_diff(g, o, c, -1, F[b], tmp);
        for (int64_t q = 0; q < N; ++q) out[a][q] -= tmp[q];
    }
}

/* Laplacian of a B-located component: sum over axes of the up/down pair of
 * first derivatives in the order its staggering requires (Sec. III, text
 * before eq:EllipticB). */
static void laplace_B(const orc_grid *g, int comp, const double *f, double *out, double *t1, double *t2)
{
    int s[3];
    int64_t N = ncells(g);
    stag_B(comp, s);
    for (int64_t q = 0; q < N; ++q) out[q] = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (s[a] == 0) { orc_diff(g, g->field_order, a, +1, f, t1); orc_diff(g, g->field_order, a, -1, t1, t2); }
        else           { orc_diff(g, g->field_order, a, -1, f, t1); orc_diff(g, g->field_order, a, +1, t1, t2); }
        for (int64_t q = 0; q < N; ++q) out[q] += t2[q];
    }
}

/* ------------------------------------------------------------------ */
/* Field gather at one position (eq:pfields, reading R6).              */
/* ------------------------------------------------------------------ */
static double gather_comp(const orc_grid *g, const double *F, const int s[3], const double xp[3])
{
    int o = g->shape_order;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        double xi = xp[a] / g->d[a];
        /* the widest support (PCS, half-integer nodes) lies in [floor-2, floor+2] */
        lo[a] = (int)floor(xi) - 2;
        hi[a] = (int)floor(xi) + 2;
    }
    double acc = 0.0;
    for (int k = lo[2]; k <= hi[2]; ++k) {
        double wz = orc_weight(o, ((k + 0.5 * s[2]) * g->d[2] - xp[2]) / g->d[2]);
        if (wz == 0.0) continue;
        for (int j = lo[1]; j <= hi[1]; ++j) {
            double wy = orc_weight(o, ((j + 0.5 * s[1]) * g->d[1] - xp[1]) / g->d[1]);
            if (wy == 0.0) continue;
            for (int i = lo[0]; i <= hi[0]; ++i) {
                double wx = orc_weight(o, ((i + 0.5 * s[0]) * g->d[0] - xp[0]) / g->d[0]);
                if (wx == 0.0) continue;
                acc += F[idx3(g, i, j, k)] * wx * wy * wz;
            }
        }
    }
    return acc;
}

void orc_gather(const orc_grid *g, double *const E[3], double *const B[3], const double xp[3],
                double Ep[3], double Bp[3])
{
    for (int a = 0; a < 3; ++a) {
        int s[3];
        stag_E(a, s);
        Ep[a] = gather_comp(g, E[a], s, xp);
        stag_B(a, s);
        Bp[a] = gather_comp(g, B[a], s, xp);
    }
}

/* ------------------------------------------------------------------ */
/* Relativistic pushers (Sec. III "Particle motion"; c = 1).           */
/* u is the proper velocity gamma*v at t - dt/2 on entry, t + dt/2 on  */
/* exit.  qmdt = q*dt/m.                                               */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Vay's pusher: the Lorentz force uses the mean of the two three-velocities;
 * the implicit equation for u(t+dt/2) has the closed-form root below (Vay 2008). */
void orc_push_vay(double qmdt, const double E[3], const double B[3], double u[3])
{
    double g0 = sqrt(1.0 + dot3(u, u));
    double tau[3] = {0.5 * qmdt * B[0], 0.5 * qmdt * B[1], 0.5 * qmdt * B[2]};
    double v0[3] = {u[0] / g0, u[1] / g0, u[2] / g0};
    double vxt[3];
    cross3(v0, tau, vxt);
    double up[3];
    for (int a = 0; a < 3; ++a) up[a] = u[a] + qmdt * E[a] + vxt[a];
    double gp2 = 1.0 + dot3(up, up);
    double ustar = dot3(up, tau);
    double tau2 = dot3(tau, tau);
    double sigma = gp2 - tau2;
    double gnew = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))));
    double t[3] = {tau[0] / gnew, tau[1] / gnew, tau[2] / gnew};
    double s = 1.0 / (1.0 + dot3(t, t));
    double upt = dot3(up, t);
    double uxt[3];
    cross3(up, t, uxt);
    for (int a = 0; a < 3; ++a) u[a] = s * (up[a] + upt * t[a] + uxt[a]);
}

/* Boris' pusher: half electric kick, magnetic rotation, half electric kick. */
void orc_push_boris(double qmdt, const double E[3], const double B[3], double u[3])
{
    double um[3];
    for (int a = 0; a < 3; ++a) um[a] = u[a] + 0.5 * qmdt * E[a];
    double gm = sqrt(1.0 + dot3(um, um));
    double t[3] = {0.5 * qmdt * B[0] / gm, 0.5 * qmdt * B[1] / gm, 0.5 * qmdt * B[2] / gm};
    double uxt[3];
    cross3(um, t, uxt);
    double uprime[3] = {um[0] + uxt[0], um[1] + uxt[1], um[2] + uxt[2]};
    double f = 2.0 / (1.0 + dot3(t, t));
    double sv[3] = {f * t[0], f * t[1], f * t[2]};
    double upxs[3];
    cross3(uprime, sv, upxs);
    for (int a = 0; a < 3; ++a) u[a] = um[a] + upxs[a] + 0.5 * qmdt * E[a];
}

/* Radiative cooling of one particle (Sec. "Radiative cooling"): um is the
 * proper velocity p- at t - dt/2, u holds p+^EM from the Lorentz push and
 * receives p+ = p+^EM + pdot_rad dt.  K = mu0 q^2 / (6 pi m c), c = 1.       */
void orc_radiate(double K, double dt, const double um[3], double u[3])
{
    double p0[3], pdot[3];
    for (int a = 0; a < 3; ++a) {
        p0[a] = 0.5 * (u[a] + um[a]);      /* time-averaged proper velocity */
        pdot[a] = (u[a] - um[a]) / dt;     /* time-centred proper acceleration */
    }
    double p2 = dot3(p0, p0);
    if (p2 == 0.0) return;
    double gamma0 = sqrt(1.0 + p2);
    double pxp[3];
    cross3(pdot, p0, pxp);
    double bracket = dot3(pdot, pdot) + dot3(pxp, pxp);   /* eq:prad over mu0 q^2 / (6 pi c) */
    double prad[3];
    for (int a = 0; a < 3; ++a) prad[a] = -K * gamma0 / p2 * bracket * p0[a];   /* eq:udot */
    for (int a = 0; a < 3; ++a) u[a] += prad[a] * dt;
}

/* ------------------------------------------------------------------ */
/* Charge-conserving deposit of one particle (Sec. III "Charge         */
/* conserving current density", eq:cc1, eq:jj3; Esirkepov 2001).       */
/* x0: position at t, x1: position at t+dt (not wrapped).              */
/* Adds q w W_a / dt to Drho[a] on the mesh (reading R2 fixes how it    */
/* is used) and the line mean data of reading R4 to lsum[a], an array   */
/* over the two transverse indices of axis a, x-fastest over them.      */
/* ------------------------------------------------------------------ */
/* old and new supports (|x1 - x0| < dx) lie in [floor(min) - 1, floor(min) + 3] */
#define ORC_SPAN 6
void orc_deposit_particle(const orc_grid *g, double q, double w, const double x0[3], const double x1[3],
                          double *Drho[3], double *lsum[3])
{
    int o = g->shape_order;
    int lo[3];
    double S0[3][ORC_SPAN], DS[3][ORC_SPAN];
    for (int a = 0; a < 3; ++a) {
        double xi0 = x0[a] / g->d[a], xi1 = x1[a] / g->d[a];
        double mn = xi0 < xi1 ? xi0 : xi1;
        lo[a] = (int)floor(mn) - 2;
        for (int m = 0; m < ORC_SPAN; ++m) {
            double xc = (lo[a] + m) * g->d[a];
            double s0 = orc_weight(o, (xc - x0[a]) / g->d[a]);
            double s1 = orc_weight(o, (xc - x1[a]) / g->d[a]);
            S0[a][m] = s0;
            DS[a][m] = s1 - s0;
        }
    }
    double qw_dt = q * w / g->dt;
    /* W_a(i,j,k) of Esirkepov: the directional share of the change of the
     * particle's charge weight on node (i,j,k). */
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int mc = 0; mc < ORC_SPAN; ++mc)
            for (int mb = 0; mb < ORC_SPAN; ++mb) {
                double tw = S0[b][mb] * S0[c][mc] + 0.5 * DS[b][mb] * S0[c][mc] +
                            0.5 * S0[b][mb] * DS[c][mc] + DS[b][mb] * DS[c][mc] / 3.0;
                if (tw == 0.0) continue;
                double moment = 0.0;
                for (int ma = 0; ma < ORC_SPAN; ++ma) {
                    double W = DS[a][ma] * tw;
                    if (W == 0.0) continue;
                    int node[3];
                    node[a] = lo[a] + ma;
                    node[b] = lo[b] + mb;
                    node[c] = lo[c] + mc;
                    Drho[a][idx3(g, node[0], node[1], node[2])] += qw_dt * W;
                    moment += (double)(lo[a] + ma) * W;
                }
                if (moment != 0.0) {
                    int tb = wrapi(lo[b] + mb, g->n[b]), tc = wrapi(lo[c] + mc, g->n[c]);
                    lsum[a][tb + (int64_t)g->n[b] * tc] += qw_dt * g->d[a] * moment;
                }
            }
    }
}

/* ------------------------------------------------------------------ */
/* Dense cyclic solve of the penta- (6th order), tri- (4th order) or   */
/* diagonal (2nd order) system of eq:penta, periodic version: entries  */
/* a+b+c on the diagonal, b+c on the first and c on the second off-   */
/* diagonals (eq:jj6d, coefficients multiplied by dx).  Gaussian        */
/* elimination with partial pivoting, one factorisation per line        */
/* length, reused for every line.                                       */
/* ------------------------------------------------------------------ */
typedef struct { int n; double *lu; int *piv; } orc_lu;

static void lu_build(orc_lu *L, int n, int order)
{
    double kc[3];
    orc_fd_coeffs(order, kc);
    double diag = kc[0] + kc[1] + kc[2], off1 = kc[1] + kc[2], off2 = kc[2];
    L->n = n;
    L->lu = (double *)calloc((size_t)n * n, sizeof(double));
    L->piv = (int *)malloc(sizeof(int) * n);
    double *A = L->lu;
    for (int r = 0; r < n; ++r) {
        A[r * n + r] += diag;
        A[r * n + wrapi(r + 1, n)] += off1;
        A[r * n + wrapi(r - 1, n)] += off1;
        A[r * n + wrapi(r + 2, n)] += off2;
        A[r * n + wrapi(r - 2, n)] += off2;
    }
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[p * n + col])) p = r;
        L->piv[col] = p;
        if (p != col)
            for (int c2 = 0; c2 < n; ++c2) { double t = A[col * n + c2]; A[col * n + c2] = A[p * n + c2]; A[p * n + c2] = t; }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r * n + col] / A[col * n + col];
            A[r * n + col] = f;
            for (int c2 = col + 1; c2 < n; ++c2) A[r * n + c2] -= f * A[col * n + c2];
        }
    }
}

static void lu_solve(const orc_lu *L, double *b)
{
    int n = L->n;
    const double *A = L->lu;
    for (int col = 0; col < n; ++col) {
        int p = L->piv[col];
        if (p != col) { double t = b[col]; b[col] = b[p]; b[p] = t; }
        for (int r = col + 1; r < n; ++r) b[r] -= A[r * n + col] * b[col];
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int c2 = r + 1; c2 < n; ++c2) acc -= A[r * n + c2] * b[c2];
        b[r] = acc / A[r * n + r];
    }
}

static void lu_free(orc_lu *L) { free(L->lu); free(L->piv); }

/* Solve one line: line[] holds -dx * D rho on input (nodes 0..n-1) and the
 * current at faces i+1/2 (stored at i) on output; mean is the line mean. */
static void current_line(const orc_lu *L, double *line, double mean)
{
    int n = L->n;
    lu_solve(L, line);                 /* line now holds Delta J_i = J(i+1/2) - J(i-1/2) */
    double run = 0.0, s = 0.0;
    for (int i = 0; i < n; ++i) { run += line[i]; line[i] = run; s += run; }  /* prefix sum */
    double c0 = mean - s / n;          /* integration constant, reading R4 */
    for (int i = 0; i < n; ++i) line[i] += c0;
}

/* Current density from the mesh-summed D rho (Sec. III, eq:jj6, eq:jj6d,
 * eq:penta), one line per transverse index pair and per component along
 * the component's own axis. */
void orc_current_from_drho(const orc_grid *g, double *const Drho[3], double *const lsum[3], double *J[3])
{
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        int n = g->n[a];
        orc_lu L;
        lu_build(&L, n, g->field_order);
        double *line = (double *)malloc(sizeof(double) * n);
        for (int tc = 0; tc < g->n[c]; ++tc)
            for (int tb = 0; tb < g->n[b]; ++tb) {
                int node[3];
                node[b] = tb;
                node[c] = tc;
                for (int i = 0; i < n; ++i) {
                    node[a] = i;
                    line[i] = -g->d[a] * Drho[a][idx3(g, node[0], node[1], node[2])];
                }
                double mean = lsum[a][tb + (int64_t)g->n[b] * tc] / n;
                current_line(&L, line, mean);
                for (int i = 0; i < n; ++i) {
                    node[a] = i;
                    J[a][idx3(g, node[0], node[1], node[2])] = line[i];
                }
            }
        free(line);
        lu_free(&L);
    }
}

/* ------------------------------------------------------------------ */
/* Implicit de-centred field update (eq:bnplus1, eq:enplus1,           */
/* eq:EllipticB with reading R3, relaxation reading R5).               */
/* E, B are advanced in place; J is J^{n+1}.                           */
/* ------------------------------------------------------------------ */
/* The explicit FDTD field update (reading R18). */
static void field_update_explicit(const orc_grid *g, double *E[3], double *B[3], double *const J[3])
{
    int64_t N = ncells(g);
    double dt = g->dt;
    double *buf = (double *)calloc((size_t)N * 4, sizeof(double));
    double *c[3] = {buf, buf + N, buf + 2 * N}, *tmp = buf + 3 * N;
    curl_plus(g, E, c, tmp);
    for (int a = 0; a < 3; ++a)
        for (int64_t q = 0; q < N; ++q) B[a][q] -= 0.5 * dt * c[a][q];
    curl_minus(g, B, c, tmp);
    for (int a = 0; a < 3; ++a)
        for (int64_t q = 0; q < N; ++q) E[a][q] += dt * (c[a][q] - J[a][q]);
    curl_plus(g, E, c, tmp);
    for (int a = 0; a < 3; ++a)
        for (int64_t q = 0; q < N; ++q) B[a][q] -= 0.5 * dt * c[a][q];
    free(buf);
}

void orc_field_update(const orc_grid *g, double *E[3], double *B[3], double *const J[3],
                      int *iters_out, double *resid_out)
{
    if (g->field_solver == 1) {
        field_update_explicit(g, E, B, J);
        if (iters_out) *iters_out = 0;
        if (resid_out) *resid_out = 0.0;
        return;
    }
    int64_t N = ncells(g);
    double alpha = g->alpha, beta = 1.0 - alpha, dt = g->dt;
    double kc[3];
    orc_fd_coeffs(g->field_order, kc);
    double kk = alpha * alpha * dt * dt;
    /* diagonal of the Laplacian stencil: -2(a^2+b^2+c^2)/dx^2 per axis */
    double l0 = 0.0;
    for (int a = 0; a < 3; ++a) l0 += -2.0 * (kc[0] * kc[0] + kc[1] * kc[1] + kc[2] * kc[2]) / (g->d[a] * g->d[a]);

    double *buf = (double *)calloc((size_t)N * 20, sizeof(double));
    double *rhs[3] = {buf, buf + N, buf + 2 * N};
    double *cE[3] = {buf + 3 * N, buf + 4 * N, buf + 5 * N};
    double *cJ[3] = {buf + 6 * N, buf + 7 * N, buf + 8 * N};
    double *Bold[3] = {buf + 9 * N, buf + 10 * N, buf + 11 * N};
    double *Bnew[3] = {buf + 12 * N, buf + 13 * N, buf + 14 * N};
    double *lap = buf + 15 * N, *t1 = buf + 16 * N, *t2 = buf + 17 * N, *tmp = buf + 18 * N;
    double *mix[3] = {cE[0], cE[1], cE[2]}; /* reused after the RHS is formed */

    curl_plus(g, E, cE, tmp);
    curl_plus(g, J, cJ, tmp);
    double rhs_max = 0.0;
    for (int a = 0; a < 3; ++a) {
        laplace_B(g, a, B[a], lap, t1, t2);
        for (int64_t q = 0; q < N; ++q) {
            rhs[a][q] = B[a][q] + alpha * beta * dt * dt * lap[q] - dt * cE[a][q] + alpha * dt * dt * cJ[a][q];
            if (fabs(rhs[a][q]) > rhs_max) rhs_max = fabs(rhs[a][q]);
            Bold[a][q] = B[a][q];
            Bnew[a][q] = B[a][q];          /* first guess B^{n+1} = B^n */
        }
    }
    /* Jacobi relaxation of (1 - alpha^2 dt^2 L) B = rhs; each sweep first
     * measures the residual of the current iterate, then updates it. */
    double *lap3[3] = {lap, t1 + 0, buf + 19 * N};
    int it = 0;
    double res = 0.0;
    for (;;) {
        res = 0.0;
        for (int a = 0; a < 3; ++a) {
            laplace_B(g, a, Bnew[a], lap3[a], tmp, t2);
            for (int64_t q = 0; q < N; ++q) {
                double r = rhs[a][q] - (Bnew[a][q] - kk * lap3[a][q]);
                if (fabs(r) > res) res = fabs(r);
            }
        }
        res = rhs_max > 0.0 ? res / rhs_max : res;
        if (res <= g->relax_tol || it >= g->relax_max_iter) break;
        for (int a = 0; a < 3; ++a)
            for (int64_t q = 0; q < N; ++q)
                Bnew[a][q] = (rhs[a][q] + kk * (lap3[a][q] - l0 * Bnew[a][q])) / (1.0 - kk * l0);
        ++it;
    }
    /* explicit E update, eq:enplus1 (c^2 mu0 = 1) */
    for (int a = 0; a < 3; ++a)
        for (int64_t q = 0; q < N; ++q) {
            B[a][q] = Bnew[a][q];
            mix[a][q] = alpha * Bnew[a][q] + beta * Bold[a][q];
        }
    double *cB[3] = {cJ[0], cJ[1], cJ[2]};
    curl_minus(g, mix, cB, tmp);
    for (int a = 0; a < 3; ++a)
        for (int64_t q = 0; q < N; ++q) E[a][q] = E[a][q] + dt * (cB[a][q] - J[a][q]);
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = res;
    free(buf);
}

/* ------------------------------------------------------------------ */
/* One leap-frog step (Sec. III, step order 1-5): for every particle   */
/* gather at x^n, push u, move, deposit; then the current solve and    */
/* the field update.  J receives J^{n+1}.                              */
/* ------------------------------------------------------------------ */
static void wrap_pos(double *x, double L)
{
    if (*x < 0.0) *x += L;
    else if (*x >= L) *x -= L;
    if (*x >= L) *x -= L;   /* x + L rounded up to L */
}

/* Direct current eq:jj2 of one particle (reading R19): adds q w v W(xm - x_c)
 * to each component on its staggered nodes. */
static void deposit_direct(const orc_grid *g, double qw, const double xm[3], const double v[3], double *J[3])
{
    int o = g->shape_order;
    for (int a = 0; a < 3; ++a) {
        int s[3];
        stag_E(a, s);
        int lo[3], hi[3];
        for (int b = 0; b < 3; ++b) {
            double xi = xm[b] / g->d[b];
            lo[b] = (int)floor(xi) - 2;
            hi[b] = (int)floor(xi) + 2;
        }
        for (int k = lo[2]; k <= hi[2]; ++k) {
            double wz = orc_weight(o, ((k + 0.5 * s[2]) * g->d[2] - xm[2]) / g->d[2]);
            if (wz == 0.0) continue;
            for (int j = lo[1]; j <= hi[1]; ++j) {
                double wy = orc_weight(o, ((j + 0.5 * s[1]) * g->d[1] - xm[1]) / g->d[1]);
                if (wy == 0.0) continue;
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    double wx = orc_weight(o, ((i + 0.5 * s[0]) * g->d[0] - xm[0]) / g->d[0]);
                    if (wx == 0.0) continue;
                    J[a][idx3(g, i, j, k)] += qw * v[a] * wx * wy * wz;
                }
            }
        }
    }
}

/* Gather, kick by kick_dt (push and cooling; none when kick_dt = 0), drift by
 * g->dt, deposit.  The plain leap-frog step has kick_dt = g->dt. */
/* One particle of a kick-drift pass: gather, push (kick), move (drift) and
 * deposit into the given arrays, then its new state. */
static void advance_particle(const orc_grid *g, double kick_dt, double *E[3], double *B[3], orc_species *P,
                             int64_t p, const double L[3], double *Drho[3], double *lsum[3], double *J[3])
{
    double qmdt = P->q * kick_dt / P->m;
    double x0[3] = {P->x[p], P->y[p], P->z[p]};
    double u[3] = {P->ux[p], P->uy[p], P->uz[p]};
    double um[3] = {u[0], u[1], u[2]};
    if (kick_dt != 0.0) {
        double Ep[3], Bp[3];
        orc_gather(g, E, B, x0, Ep, Bp);
        if (g->pusher == 1) orc_push_boris(qmdt, Ep, Bp, u);
        else orc_push_vay(qmdt, Ep, Bp, u);
        if (P->rad != 0.0) orc_radiate(P->rad, kick_dt, um, u);
    }
    double gam = sqrt(1.0 + dot3(u, u));
    double x1[3];
    for (int a = 0; a < 3; ++a) x1[a] = x0[a] + g->dt * u[a] / gam;
    if (g->current_mode == 1) {
        double xm[3], v[3];
        for (int a = 0; a < 3; ++a) {
            xm[a] = 0.5 * (x0[a] + x1[a]);
            v[a] = u[a] / gam;
        }
        deposit_direct(g, P->q * P->w, xm, v, J);
    } else {
        orc_deposit_particle(g, P->q, P->w, x0, x1, Drho, lsum);
    }
    wrap_pos(&x1[0], L[0]);
    wrap_pos(&x1[1], L[1]);
    wrap_pos(&x1[2], L[2]);
    P->x[p] = x1[0]; P->y[p] = x1[1]; P->z[p] = x1[2];
    P->ux[p] = u[0]; P->uy[p] = u[1]; P->uz[p] = u[2];
}

/* Threads of the particle loop: 1 unless set (an OpenMP build only), used
 * for the all-core timing baseline.  As in the paper's Sec. IX OpenMP level,
 * each thread deposits into its own copies of the charge-change (or direct
 * current) and line-sum arrays, and the copies are added after the loop; with
 * one thread the sums are those of the plain loop, bit for bit. */
static int orc_threads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    orc_threads = n < 1 ? 1 : n;
#else
    (void)n;
    orc_threads = 1;
#endif
    return orc_threads;
}

void orc_particles_kick_drift(const orc_grid *g, double kick_dt, double *E[3], double *B[3], orc_species *sp,
                              int nsp, double *J[3])
{
    int64_t N = ncells(g);
    int64_t nl[3];
    double *Drho[3], *lsum[3];
    for (int a = 0; a < 3; ++a) {
        Drho[a] = (double *)calloc((size_t)N, sizeof(double));
        int b = (a + 1) % 3, c = (a + 2) % 3;
        nl[a] = (int64_t)g->n[b] * g->n[c];
        lsum[a] = (double *)calloc((size_t)nl[a], sizeof(double));
    }
    double L[3] = {g->n[0] * g->d[0], g->n[1] * g->d[1], g->n[2] * g->d[2]};
    if (g->current_mode == 1)
        for (int a = 0; a < 3; ++a) memset(J[a], 0, sizeof(double) * (size_t)N);
    const int nt = orc_threads;
    /* per-thread copies: Drho (or J for the direct current) and lsum */
    double **tbuf = (double **)calloc((size_t)nt * 6, sizeof(double *));
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            tbuf[6 * t + a] = (double *)calloc((size_t)N, sizeof(double));
            tbuf[6 * t + 3 + a] = (double *)calloc((size_t)nl[a], sizeof(double));
        }
    for (int s = 0; s < nsp; ++s) {
        orc_species *P = &sp[s];
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
        for (int64_t p = 0; p < P->n; ++p) {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            double *dr[3] = {tbuf[6 * t], tbuf[6 * t + 1], tbuf[6 * t + 2]};
            double *ls[3] = {tbuf[6 * t + 3], tbuf[6 * t + 4], tbuf[6 * t + 5]};
            advance_particle(g, kick_dt, E, B, P, p, L, dr, ls, dr);
        }
    }
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            double *dst = g->current_mode == 1 ? J[a] : Drho[a];
            for (int64_t i = 0; i < N; ++i) dst[i] += tbuf[6 * t + a][i];
            for (int64_t i = 0; i < nl[a]; ++i) lsum[a][i] += tbuf[6 * t + 3 + a][i];
            free(tbuf[6 * t + a]);
            free(tbuf[6 * t + 3 + a]);
        }
    free(tbuf);
    if (g->current_mode != 1) orc_current_from_drho(g, Drho, lsum, J);
    for (int a = 0; a < 3; ++a) { free(Drho[a]); free(lsum[a]); }
}

void orc_particles_deposit(const orc_grid *g, double *E[3], double *B[3], orc_species *sp, int nsp,
                           double *J[3])
{
    orc_particles_kick_drift(g, g->dt, E, B, sp, nsp, J);
}

void orc_step(const orc_grid *g, double *E[3], double *B[3], double *J[3], orc_species *sp, int nsp,
              int *iters_out, double *resid_out)
{
    orc_particles_deposit(g, E, B, sp, nsp, J);
    orc_field_update(g, E, B, J, iters_out, resid_out);
}

/* Kick (b) and drift (a) fractions of the four substeps of reading R17. */
void orc_step4_coeffs(double a[4], double b[4])
{
    double w1 = 1.0 / (2.0 - cbrt(2.0));
    double w0 = -cbrt(2.0) * w1;
    a[0] = a[3] = 0.5 * w1;
    a[1] = a[2] = 0.5 * (w0 + w1);
    b[0] = 0.0;
    b[1] = b[3] = w1;
    b[2] = w0;
}

/* One 4th-order step (reading R17): four kick-drift substeps, each followed by
 * the field update over its drift. */
void orc_step4(const orc_grid *g, double *E[3], double *B[3], double *J[3], orc_species *sp, int nsp,
               int *iters_out, double *resid_out)
{
    double a[4], b[4];
    orc_step4_coeffs(a, b);
    for (int i = 0; i < 4; ++i) {
        orc_grid sub = *g;
        sub.dt = a[i] * g->dt;
        orc_particles_kick_drift(&sub, b[i] * g->dt, E, B, sp, nsp, J);
        orc_field_update(&sub, E, B, J, iters_out, resid_out);
    }
}

/* ------------------------------------------------------------------ */
/* Charge density on the integer nodes (eq:rho2).                      */
/* ------------------------------------------------------------------ */
void orc_rho(const orc_grid *g, const orc_species *sp, int nsp, double *rho)
{
    int64_t N = ncells(g);
    for (int64_t q = 0; q < N; ++q) rho[q] = 0.0;
    int o = g->shape_order;
    for (int s = 0; s < nsp; ++s) {
        const orc_species *P = &sp[s];
        for (int64_t p = 0; p < P->n; ++p) {
            double xp[3] = {P->x[p], P->y[p], P->z[p]};
            int lo[3];
            for (int a = 0; a < 3; ++a) lo[a] = (int)floor(xp[a] / g->d[a]) - 3;
            for (int k = lo[2]; k <= lo[2] + 6; ++k) {
                double wz = orc_weight(o, (k * g->d[2] - xp[2]) / g->d[2]);
                if (wz == 0.0) continue;
                for (int j = lo[1]; j <= lo[1] + 6; ++j) {
                    double wy = orc_weight(o, (j * g->d[1] - xp[1]) / g->d[1]);
                    if (wy == 0.0) continue;
                    for (int i = lo[0]; i <= lo[0] + 6; ++i) {
                        double wx = orc_weight(o, (i * g->d[0] - xp[0]) / g->d[0]);
                        if (wx == 0.0) continue;
                        rho[idx3(g, i, j, k)] += P->q * P->w * wx * wy * wz;
                    }
                }
            }
        }
    }
}

/* div^- of an E-located (face) vector: the discrete Gauss operator. */
void orc_div_minus(const orc_grid *g, double *const F[3], double *out)
{
    int64_t N = ncells(g);
    double *t = (double *)malloc(sizeof(double) * N);
    for (int64_t q = 0; q < N; ++q) out[q] = 0.0;
    for (int a = 0; a < 3; ++a) {
        orc_diff(g, g->field_order, a, -1, F[a], t);
        for (int64_t q = 0; q < N; ++q) out[q] += t[q];
    }
    free(t);
}

/* div^+ of a B-located (edge) vector, at cell corners. */
void orc_div_plus(const orc_grid *g, double *const F[3], double *out)
{
    int64_t N = ncells(g);
    double *t = (double *)malloc(sizeof(double) * N);
    for (int64_t q = 0; q < N; ++q) out[q] = 0.0;
    for (int a = 0; a < 3; ++a) {
        orc_diff(g, g->field_order, a, +1, F[a], t);
        for (int64_t q = 0; q < N; ++q) out[q] += t[q];
    }
    free(t);
}

/* Divergence filter (reading R20): `passes` simultaneous smoothing steps of E
 * towards div^- E = rho and of B towards div^+ B = 0. */
void orc_divergence_filter(const orc_grid *g, double *E[3], double *B[3], const double *rho, int passes)
{
    int64_t N = ncells(g);
    double kc[3];
    orc_fd_coeffs(g->field_order, kc);
    double lam = 0.0;   /* max over wave numbers of sum_a K_a^2 */
    for (int a = 0; a < 3; ++a) {
        double best = 0.0;
        for (int s = 0; s <= 4000; ++s) {
            double th = 3.14159265358979323846 * s / 4000.0;
            double K = (2.0 / g->d[a]) * (kc[0] * sin(0.5 * th) + kc[1] * sin(1.5 * th) + kc[2] * sin(2.5 * th));
            if (K * K > best) best = K * K;
        }
        lam += best;
    }
    double tau = 1.0 / lam;
    double *r = (double *)malloc(sizeof(double) * (size_t)N), *d = (double *)malloc(sizeof(double) * (size_t)N);
    for (int p = 0; p < passes; ++p) {
        orc_div_minus(g, E, r);
        for (int64_t q = 0; q < N; ++q) r[q] -= rho[q];
        for (int a = 0; a < 3; ++a) {
            orc_diff(g, g->field_order, a, +1, r, d);
            for (int64_t q = 0; q < N; ++q) E[a][q] += tau * d[q];
        }
        orc_div_plus(g, B, r);
        for (int a = 0; a < 3; ++a) {
            orc_diff(g, g->field_order, a, -1, r, d);
            for (int64_t q = 0; q < N; ++q) B[a][q] += tau * d[q];
        }
    }
    free(r);
    free(d);
}

/* Global diagnostics (energies, total charge, Gauss and div B residuals). */
void orc_diagnostics(const orc_grid *g, double *const E[3], double *const B[3], const orc_species *sp, int nsp,
                     orc_diag *out)
{
    int64_t N = ncells(g);
    double dV = g->d[0] * g->d[1] * g->d[2];
    double *rho = (double *)malloc(sizeof(double) * N);
    double *dv = (double *)malloc(sizeof(double) * N);
    memset(out, 0, sizeof(*out));
    for (int64_t q = 0; q < N; ++q) {
        double e2 = E[0][q] * E[0][q] + E[1][q] * E[1][q] + E[2][q] * E[2][q];
        double b2 = B[0][q] * B[0][q] + B[1][q] * B[1][q] + B[2][q] * B[2][q];
        out->energy_E += 0.5 * e2 * dV;
        out->energy_B += 0.5 * b2 * dV;
        out->energy_Ex += 0.5 * E[0][q] * E[0][q] * dV;
    }
    for (int s = 0; s < nsp; ++s)
        for (int64_t p = 0; p < sp[s].n; ++p) {
            double u2 = sp[s].ux[p] * sp[s].ux[p] + sp[s].uy[p] * sp[s].uy[p] + sp[s].uz[p] * sp[s].uz[p];
            out->kinetic += sp[s].w * dV * sp[s].m * (sqrt(1.0 + u2) - 1.0);
        }
    orc_rho(g, sp, nsp, rho);
    orc_div_minus(g, E, dv);
    for (int64_t q = 0; q < N; ++q) {
        out->charge += rho[q] * dV;
        double gq = fabs(dv[q] - rho[q]);
        if (gq > out->gauss_max) out->gauss_max = gq;
        if (fabs(rho[q]) > out->rho_max) out->rho_max = fabs(rho[q]);
    }
    orc_div_plus(g, B, dv);
    for (int64_t q = 0; q < N; ++q)
        if (fabs(dv[q]) > out->divB_max) out->divB_max = fabs(dv[q]);
    free(rho);
    free(dv);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random        */
/* numbers: as easy as 1, 2, 3", SC'11): ten rounds of                 */
/*   (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2),             */
/*                        hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))              */
/* with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key bumped by the Weyl   */
/* constants (0x9E3779B9, 0xBB67AE85) between rounds.  Reading R23.    */
/* ------------------------------------------------------------------ */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x[1] ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x[3] ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
    }
    for (int m = 0; m < 4; ++m) out[m] = x[m];
}

/* n draws of four uniforms in (0, 1): draw i is Philox of counter
 * (i, 0, step, stream) under key (seed low, seed high), each word r mapped to
 * (r + 1/2) 2^-32.  out holds 4 n values. */
void orc_draws(uint64_t seed, uint32_t step, uint32_t stream, int64_t n, double *out)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t ctr[4] = {(uint32_t)i, 0u, step, stream};
        uint32_t r[4];
        orc_philox4x32(ctr, key, r);
        for (int m = 0; m < 4; ++m) out[4 * i + m] = ((double)r[m] + 0.5) * (1.0 / 4294967296.0);
    }
}
