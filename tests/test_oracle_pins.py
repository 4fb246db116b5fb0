"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, exact invariants, brute force on tiny inputs, or an
independent (spectral) solution of the defining equations.  A plausible slip in
the oracle (a dropped term, a wrong sign, index or staggering, a transposed
operand, the printed 6th-order coefficient) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from tests import theory

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(v) for v in line.split()])
    return rows


# --------------------------------------------------------------------------
# Weight functions (Sec. II)
# --------------------------------------------------------------------------

def test_weight_golden_values(orc):
    for order, delta, w in _golden("weights.txt"):
        assert orc.weight(int(order), delta) == pytest.approx(w, abs=1e-15), (order, delta)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_weight_partition_of_unity_and_linear_reproduction(orc, order):
    rng = np.random.default_rng(5)
    for xi in rng.random(200) * 10.0 + 3.0:
        nodes = np.arange(int(xi) - 4, int(xi) + 6)
        w = np.array([orc.weight(order, i - xi) for i in nodes])
        assert w.min() >= 0.0
        if order == 0 and abs((xi % 1.0) - 0.5) < 1e-12:
            continue
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        if order >= 1:
            assert (nodes * w).sum() == pytest.approx(xi, abs=1e-12)
        assert np.count_nonzero(w) <= order + 1


@pytest.mark.parametrize("order", [1, 2, 3])
def test_weight_continuity_symmetry_and_unit_integral(orc, order):
    half = (order + 1) / 2.0
    breaks = np.arange(-half, half + 1e-9, 1.0)
    for b in breaks:
        lo, hi = orc.weight(order, b - 1e-9), orc.weight(order, b + 1e-9)
        assert lo == pytest.approx(hi, abs=1e-8)
    xs = np.linspace(-3, 3, 60001)
    w = np.array([orc.weight(order, x) for x in xs])
    assert np.allclose(w, w[::-1], atol=1e-15)
    assert np.trapezoid(w, xs) == pytest.approx(1.0, abs=1e-7)


# --------------------------------------------------------------------------
# Staggered difference operators (Sec. III)
# --------------------------------------------------------------------------

def test_fd_coefficients_printed_and_taylor(orc):
    for order, a, b, c in _golden("fd_coeffs.txt"):
        k = orc.fd_coeffs(int(order))
        assert np.allclose(k, [a, b, c], atol=1e-16)
        assert k[0] + 3 * k[1] + 5 * k[2] == pytest.approx(1.0, abs=1e-15)
        if order >= 4:
            assert k[0] + 27 * k[1] + 125 * k[2] == pytest.approx(0.0, abs=1e-14)
        if order >= 6:
            assert k[0] + 243 * k[1] + 3125 * k[2] == pytest.approx(0.0, abs=1e-13)
    # the printed 25/21 violates the first condition
    assert 25 / 21 + 3 * (-25 / 384) + 5 * (3 / 640) == pytest.approx(1.0186, abs=1e-4)


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fd_convergence_order(orc, order, axis):
    """d^+ and d^- of sin(2 pi x / L) converge at the stated order, on the
    staggered positions (a half-cell offset error would show as 1st order)."""
    errs = {+1: [], -1: []}
    for n in (16, 32):
        shape = [4, 4, 4]
        shape[axis] = n
        d = [0.3, 0.3, 0.3]
        d[axis] = 1.0 / n
        g = orc.make_grid(shape, d, 0.1)
        x = np.arange(n) * d[axis]
        for direction in (+1, -1):
            xin = x if direction > 0 else x + 0.5 * d[axis]     # sample positions of the input
            xout = x + 0.5 * d[axis] if direction > 0 else x    # positions of the result
            f1 = np.sin(2 * np.pi * xin)
            exp1 = 2 * np.pi * np.cos(2 * np.pi * xout)
            sh = [1, 1, 1]
            sh[2 - axis] = n
            f = np.broadcast_to(f1.reshape(sh), (shape[2], shape[1], shape[0])).copy()
            out = orc.diff(g, f, axis, direction, order)
            e = np.abs(out - np.broadcast_to(exp1.reshape(sh), out.shape)).max()
            errs[direction].append(e)
    for direction in (+1, -1):
        rate = math.log2(errs[direction][0] / errs[direction][1])
        assert rate == pytest.approx(order, abs=0.15), (direction, errs[direction])


def test_div_of_curl_vanishes(orc):
    g = orc.make_grid((6, 5, 4), (0.5, 0.4, 0.3), 0.1)
    rng = np.random.default_rng(1)
    F = [rng.standard_normal((4, 5, 6)) for _ in range(3)]

    def curl(F, direction):
        out = []
        for a in range(3):
            b, c = (a + 1) % 3, (a + 2) % 3
            out.append(orc.diff(g, F[c], b, direction) - orc.diff(g, F[b], c, direction))
        return out

    assert np.abs(orc.div_plus(g, curl(F, +1))).max() < 1e-12
    assert np.abs(orc.div_minus(g, curl(F, -1))).max() < 1e-12


# --------------------------------------------------------------------------
# Gather (eq:pfields)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [1, 2, 3])
def test_gather_uniform_and_linear_fields(orc, shape):
    n = (12, 12, 12)
    d = (0.5, 0.4, 0.3)
    g = orc.make_grid(n, d, 0.1, shape_order=shape)
    z, y, x = np.meshgrid(np.arange(12.0), np.arange(12.0), np.arange(12.0), indexing="ij")
    idx = (x, y, z)
    # E_a linear in its own coordinate, sampled at its staggered node (i+1/2);
    # B_a linear in the next coordinate, sampled at half-integer positions there.
    E = [(idx[a] + 0.5) * d[a] for a in range(3)]
    B = [(idx[(a + 1) % 3] + 0.5) * d[(a + 1) % 3] for a in range(3)]
    rng = np.random.default_rng(3)
    for _ in range(20):
        xp = (4.0 + 3.0 * rng.random(3)) * np.array(d)   # away from the periodic seam
        Ep, Bp = orc.gather(g, E, B, xp)
        for a in range(3):
            assert Ep[a] == pytest.approx(xp[a], abs=1e-12)
            assert Bp[a] == pytest.approx(xp[(a + 1) % 3], abs=1e-12)
        Ec = [np.full((12, 12, 12), v) for v in (1.5, -2.0, 0.25)]
        Ep, Bp = orc.gather(g, Ec, Ec, xp)
        assert np.allclose(Ep, [1.5, -2.0, 0.25], atol=1e-14)


# --------------------------------------------------------------------------
# Pushers (Sec. III "Particle motion")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pusher", [0, 1])
def test_pure_B_gyration_closes(orc, pusher):
    u0 = np.array([0.8, 0.0, 0.3])
    g0 = math.sqrt(1 + u0 @ u0)
    dt, q, m = 0.2, -1.0, 1.0
    Bz = 2 * m * g0 * math.tan(math.pi / 64) / (abs(q) * dt)   # rotation 2*pi/64 per step
    u = u0.copy()
    for _ in range(64):
        u = orc.push(q * dt / m, [0, 0, 0], [0, 0, Bz], u, pusher)
        assert math.sqrt(u @ u) == pytest.approx(math.sqrt(u0 @ u0), rel=1e-14)
    assert np.allclose(u, u0, atol=1e-13)
    # a quarter orbit turns u_perp by 90 degrees about -z for an electron in +B_z
    u = u0.copy()
    for _ in range(16):
        u = orc.push(q * dt / m, [0, 0, 0], [0, 0, Bz], u, pusher)
    assert np.allclose(u, [0.0, 0.8, 0.3], atol=1e-13)


@pytest.mark.parametrize("pusher", [0, 1])
def test_pure_E_kick(orc, pusher):
    u = np.array([0.1, -0.2, 0.05])
    E = np.array([0.3, 0.7, -0.4])
    qmdt = -0.25
    for _ in range(10):
        u_new = orc.push(qmdt, E, [0, 0, 0], u, pusher)
        assert np.allclose(u_new - u, qmdt * E, atol=1e-15)
        u = u_new


def test_ExB_drift_vay_exact_boris_not(orc):
    E = np.array([0.0, 0.6, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    vD = np.cross(E, B) / (B @ B)
    gD = 1 / math.sqrt(1 - vD @ vD)
    u0 = gD * vD
    u_v, u_b = u0.copy(), u0.copy()
    for _ in range(50):
        u_v = orc.push(-0.1, E, B, u_v, 0)
        u_b = orc.push(-0.1, E, B, u_b, 1)
    assert np.abs(u_v - u0).max() < 1e-13        # Vay: force-free drift is a fixed point
    assert np.abs(u_b - u0).max() > 1e-4         # Boris: known spurious force


# --------------------------------------------------------------------------
# Charge-conserving deposit and high-order current (eq:cc1 .. eq:penta)
# --------------------------------------------------------------------------

def _one_particle(orc, shape, forder, x0, u, n=(8, 8, 8), d=(0.5, 0.4, 0.3), dt=0.1, q=-1.0, w=0.7):
    sim = orc.Simulation(n, d, dt, field_order=forder, shape_order=shape)
    sim.add_species(q, 1.0, w, [x0[0]], [x0[1]], [x0[2]], [u[0]], [u[1]], [u[2]])
    rho0 = sim.rho()
    sim.deposit()
    rho1 = sim.rho()
    sp = sim.species[0]
    x1 = np.array([sp["x"][0], sp["y"][0], sp["z"][0]])
    return sim, rho0, rho1, x1


CASES = [((1.3, 1.7, 0.9), (0.4, -0.3, 0.2)),
         ((3.99, 0.01, 2.2), (2.0, -2.5, 0.0)),      # crosses cell faces on two axes
         ((0.05, 3.15, 0.02), (-1.5, 1.2, -3.0))]     # crosses the periodic seam


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("forder", [2, 4, 6])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_single_particle_continuity(orc, shape, forder, case):
    x0, u = CASES[case]
    sim, rho0, rho1, x1 = _one_particle(orc, shape, forder, x0, u)
    dt = sim.g.dt
    drho = (rho1 - rho0) / dt
    res = drho + orc.div_minus(sim.g, sim.J)
    assert np.abs(res).max() <= 1e-13 * np.abs(drho).max()


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("forder", [2, 4, 6])
def test_single_particle_total_current(orc, shape, forder):
    """Sum over cells of J_a equals q w (x1_a - x0_a)/dt (B-spline linear
    reproduction), independent of the field order (the solve keeps the mean)."""
    n, d, dt, q, w = (8, 8, 8), (0.5, 0.4, 0.3), 0.1, -1.0, 0.7
    for x0, u in CASES:
        sim, _, _, x1 = _one_particle(orc, shape, forder, x0, u, n, d, dt, q, w)
        gam = math.sqrt(1 + np.dot(u, u))
        # the particle's unwrapped displacement is dt * v
        for a in range(3):
            disp = dt * u[a] / gam
            assert sim.J[a].sum() == pytest.approx(q * w * disp / dt, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_motion_along_x_only_and_at_rest(orc, shape):
    sim, _, _, _ = _one_particle(orc, shape, 6, (1.3, 1.7, 0.9), (0.9, 0.0, 0.0))
    assert np.abs(sim.J[1]).max() == 0.0 and np.abs(sim.J[2]).max() == 0.0
    assert np.abs(sim.J[0]).max() > 0.0
    sim, _, _, _ = _one_particle(orc, shape, 6, (1.3, 1.7, 0.9), (0.0, 0.0, 0.0))
    assert max(np.abs(sim.J[a]).max() for a in range(3)) == 0.0


def test_cic_textbook_current(orc):
    """CIC moving along x inside one cell, 2nd-order fields: the only current is
    J_x on the face the particle sits on, q w v_x times the fixed transverse
    CIC weights (the classic area-weighting result)."""
    d, dt, q, w = (0.5, 0.4, 0.3), 0.1, -1.0, 0.7
    x0 = (1.1, 1.7, 0.9)
    u = (0.5, 0.0, 0.0)
    sim, _, _, x1 = _one_particle(orc, 1, 2, x0, u, d=d, dt=dt, q=q, w=w)
    vx = u[0] / math.sqrt(1 + u[0] ** 2)
    assert int(x1[0] / d[0]) == int(x0[0] / d[0])
    eta, zeta = x0[1] / d[1], x0[2] / d[2]
    j0, k0 = int(eta), int(zeta)
    expect = np.zeros((8, 8, 8))
    for j, wy in ((j0, 1 - (eta - j0)), (j0 + 1, eta - j0)):
        for k, wz in ((k0, 1 - (zeta - k0)), (k0 + 1, zeta - k0)):
            expect[k, j, int(x0[0] / d[0])] = q * w * vx * wy * wz
    assert np.allclose(sim.J[0], expect, atol=1e-14)


@pytest.mark.parametrize("forder", [4, 6])
def test_high_order_current_brute_force(orc, forder):
    """J of order 4/6 for one particle equals the dense least-squares solution
    of  d^-_{order} J = d^-_2 J_2  (both equal -D rho) with the line mean of the
    2nd-order current J_2 (reading R4); the dense operator is assembled by
    applying the oracle's own difference to unit vectors, independently of the
    banded solve and prefix sum being checked."""
    x0, u = CASES[1]
    n = (8, 8, 8)
    sim2, _, _, _ = _one_particle(orc, 3, 2, x0, u, n)
    simh, _, _, _ = _one_particle(orc, 3, forder, x0, u, n)
    g = simh.g
    N = n[0]
    D = np.zeros((N, N))
    for i in range(N):
        e = np.zeros((1, 1, N))
        e[0, 0, i] = 1.0
        gg = orc.make_grid((N, 1, 1), (g.d[0], 1, 1), g.dt, field_order=forder)
        D[:, i] = orc.diff(gg, e, 0, -1, forder)[0, 0]
    D2 = np.zeros((N, N))
    for i in range(N):
        e = np.zeros((1, 1, N))
        e[0, 0, i] = 1.0
        gg = orc.make_grid((N, 1, 1), (g.d[0], 1, 1), g.dt, field_order=2)
        D2[:, i] = orc.diff(gg, e, 0, -1, 2)[0, 0]
    for k in range(n[2]):
        for j in range(n[1]):
            J2 = sim2.J[0][k, j]
            rhs = D2 @ J2
            A = np.vstack([D, np.ones((1, N))])
            b = np.concatenate([rhs, [J2.sum()]])
            sol, *_ = np.linalg.lstsq(A, b, rcond=None)
            assert np.allclose(simh.J[0][k, j], sol, atol=1e-13)


# --------------------------------------------------------------------------
# Implicit field update (eq:bnplus1, eq:enplus1, eq:EllipticB)
# --------------------------------------------------------------------------

def _symbols(g, order):
    """Fourier symbols of d^+ and d^- per axis for arrays of shape (nz, ny, nx)."""
    k3 = np.array(order)
    kc = {6: (75 / 64, -25 / 384, 3 / 640), 4: (9 / 8, -1 / 24, 0.0), 2: (1.0, 0.0, 0.0)}[order]
    Dp, Dm = [], []
    for a in range(3):
        n, h = g.n[a], g.d[a]
        k = 2 * np.pi * np.fft.fftfreq(n, d=h)
        K = (2 / h) * sum(kc[m] * np.sin((2 * m + 1) * k * h / 2) for m in range(3))
        sh = [1, 1, 1]
        sh[2 - a] = n
        Dp.append((1j * K * np.exp(+0.5j * k * h)).reshape(sh))
        Dm.append((1j * K * np.exp(-0.5j * k * h)).reshape(sh))
    del k3
    return Dp, Dm


def _curl_matrix(D):
    Z = np.zeros(np.broadcast(D[0], D[1], D[2]).shape, dtype=complex)
    Dx, Dy, Dz = [np.broadcast_to(v, Z.shape) for v in D]
    return np.array([[Z, -Dz, Dy], [Dz, Z, -Dx], [-Dy, Dx, Z]])


@pytest.mark.parametrize("order", [2, 4, 6])
def test_field_update_equals_direct_solve_of_defining_equations(orc, order):
    """The oracle's relaxed elliptic form equals a per-Fourier-mode direct solve
    of the two defining equations eq:bnplus1 / eq:enplus1 (6x6 complex system),
    which pins the derivation of eq:EllipticB, including the sign of its
    current term (reading R3)."""
    n, d, dt, alpha = (6, 5, 4), (0.5, 0.4, 0.3), 0.12, 0.6
    g = orc.make_grid(n, d, dt, field_order=order, alpha=alpha, relax_tol=1e-15, relax_max_iter=500)
    rng = np.random.default_rng(11)
    shp = (n[2], n[1], n[0])
    E = [rng.standard_normal(shp) for _ in range(3)]
    J = [rng.standard_normal(shp) for _ in range(3)]
    A = [rng.standard_normal(shp) for _ in range(3)]
    B = [orc.diff(g, A[(a + 2) % 3], (a + 1) % 3, +1) - orc.diff(g, A[(a + 1) % 3], (a + 2) % 3, +1)
         for a in range(3)]                         # B = curl^+ A, divergence-free
    E0 = [e.copy() for e in E]
    B0 = [b.copy() for b in B]
    orc.field_update(g, E, B, J)

    Dp, Dm = _symbols(g, order)
    Cp, Cm = _curl_matrix(Dp), _curl_matrix(Dm)
    f = lambda L: np.array([np.fft.fftn(v) for v in L])
    Eh, Bh, Jh = f(E0), f(B0), f(J)
    beta = 1 - alpha
    I3 = np.eye(3)[:, :, None, None, None] * np.ones(shp)
    # unknowns [B1; E1]:  B1 + a dt C+ E1 = B0 - b dt C+ E0 ;  -a dt C- B1 + E1 = E0 + b dt C- B0 - dt J
    M = np.zeros((6, 6) + shp, dtype=complex)
    M[:3, :3] = I3
    M[:3, 3:] = alpha * dt * Cp
    M[3:, :3] = -alpha * dt * Cm
    M[3:, 3:] = I3
    rhsB = Bh - beta * dt * np.einsum("ij...,j...->i...", Cp, Eh)
    rhsE = Eh + beta * dt * np.einsum("ij...,j...->i...", Cm, Bh) - dt * Jh
    rhs = np.concatenate([rhsB, rhsE])
    Mt = np.moveaxis(M, (0, 1), (-2, -1))
    sol = np.linalg.solve(Mt, np.moveaxis(rhs, 0, -1)[..., None])[..., 0]
    sol = np.moveaxis(sol, -1, 0)
    B1 = [np.fft.ifftn(sol[a]).real for a in range(3)]
    E1 = [np.fft.ifftn(sol[3 + a]).real for a in range(3)]
    scale = max(np.abs(v).max() for v in B1 + E1)
    for a in range(3):
        assert np.abs(B[a] - B1[a]).max() < 1e-12 * scale
        assert np.abs(E[a] - E1[a]).max() < 1e-12 * scale
    assert np.abs(orc.div_plus(g, B)).max() < 1e-12 * scale


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("mode", [1, 3, 6])
def test_vacuum_mode_damping_closed_form(orc, order, mode):
    """A vacuum plane wave loses energy per step by the closed-form factor of
    the theta-scheme, |G|^2 = (1 + beta^2 s^2)/(1 + alpha^2 s^2), s = dt K(k)."""
    nx, dx, dt, alpha = 16, 0.5, 0.25, 0.55
    g = orc.make_grid((nx, 2, 2), (dx, dx, dx), dt, field_order=order, alpha=alpha, relax_tol=1e-15,
                      relax_max_iter=500)
    k = 2 * np.pi * mode / (nx * dx)
    kc = orc.fd_coeffs(order)
    K = (2 / dx) * (kc[0] * np.sin(k * dx / 2) + kc[1] * np.sin(3 * k * dx / 2) + kc[2] * np.sin(5 * k * dx / 2))
    s = dt * K
    ratio = (1 + (1 - alpha) ** 2 * s * s) / (1 + alpha ** 2 * s * s)
    x = np.arange(nx) * dx
    E = [np.zeros((2, 2, nx)) for _ in range(3)]
    B = [np.zeros((2, 2, nx)) for _ in range(3)]
    J = [np.zeros((2, 2, nx)) for _ in range(3)]
    E[1][...] = np.cos(k * x)
    B[2][...] = 0.3 * np.sin(k * (x + dx / 2))
    W0 = sum((v ** 2).sum() for v in E + B)
    for _ in range(3):
        orc.field_update(g, E, B, J)
        W1 = sum((v ** 2).sum() for v in E + B)
        assert W1 / W0 == pytest.approx(ratio, rel=1e-12)
        W0 = W1


# --------------------------------------------------------------------------
# Whole-step invariants and physics
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,forder", [(2, 6), (3, 6), (3, 4), (1, 2)])
def test_gauss_and_divB_invariants_over_steps(orc, shape, forder):
    import pp_synth
    L = pp_synth.thermal(n=(8, 6, 5), ppc=2, u_th=0.3, dx=0.5, dt=0.25, seed=7)
    sim = orc.Simulation(L.n, L.d, L.dt, field_order=forder, shape_order=shape, relax_tol=1e-14)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    d0 = sim.diagnostics()
    assert d0["gauss_max"] < 1e-14 and abs(d0["charge"]) < 1e-14
    for _ in range(6):
        sim.step(1)
        d = sim.diagnostics()
        assert d["gauss_max"] < 1e-12 * max(d["rho_max"], 1e-300)
        assert d["divB_max"] < 1e-12
        assert abs(d["charge"]) < 1e-13
        assert d["relax_residual"] <= 1e-14


@pytest.mark.parametrize("mode,shape", [(2, 2), (3, 3)])
def test_quiet_two_stream_growth_matches_cold_theory(orc, mode, shape):
    """Quiet-start cold pair two-stream: the energy in E_x grows at twice the
    closed-form cold growth rate (relativistic longitudinal mass Gamma^3)."""
    import pp_synth
    L = pp_synth.quiet_two_stream(nx=32, dx=0.25, dt=0.125, mode=mode)
    sim = orc.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=shape, relax_tol=1e-13)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    nst = 240
    W = []
    for _ in range(nst):
        sim.step(1)
        W.append(sim.diagnostics()["energy_Ex"])
    t = np.arange(1, nst + 1) * L.dt
    rate, npts = theory.fit_growth(t, W)
    expect = theory.cold_two_stream(L.params["k"], L.params["beta"])
    assert npts >= 40
    assert rate == pytest.approx(expect, rel=0.03)


def test_bret_growth_formulas_reproduce_printed_values():
    (mmi, fi, tsi), = _golden("bret_growth.txt")
    assert theory.bret_mmi(0.1, 4.0) == pytest.approx(mmi, abs=6e-4)
    assert theory.bret_fi(0.1, 4.0) == pytest.approx(fi, abs=6e-4)
    assert theory.bret_tsi(0.1, 4.0) == pytest.approx(tsi, abs=6e-4)
    # the other reading of alpha misses the printed MMI value in the third digit
    assert abs(theory.bret_mmi(0.1 / 0.9, 4.0) - mmi) > 5e-3


def test_cold_two_stream_closed_form_values():
    beta = 0.2
    ks = [2 * np.pi * m / 8.0 for m in (4, 5, 6)]
    got = [theory.cold_two_stream(k, beta) for k in ks]
    assert np.allclose(got, [0.452, 0.483, 0.477], atol=1.5e-3)


# --------------------------------------------------------------------------
# Radiative cooling (Sec. "Radiative cooling", eq:prad, eq:udot)
# --------------------------------------------------------------------------

def _synchrotron_gamma(orc, dt, pusher, T=45.0, K=0.01, g0=10.0, q=-1.0, m=1.0, B=1.0):
    u = np.array([math.sqrt(g0 * g0 - 1.0), 0.0, 0.0])
    n = int(round(T / dt))
    for _ in range(n):
        um = u.copy()
        u = orc.push(q * dt / m, [0.0, 0.0, 0.0], [0.0, 0.0, B], u, pusher)
        u = orc.radiate(K, dt, um, u)
    # closed form: gamma' = -kappa (gamma^2 - 1), kappa = K (q/m)^2 B^2, so
    # (gamma - 1)/(gamma + 1) decays as exp(-2 kappa t)
    kappa = K * (q / m) ** 2 * B * B
    C = (g0 - 1.0) / (g0 + 1.0) * math.exp(-2.0 * kappa * n * dt)
    exact = (1.0 + C) / (1.0 - C)
    return math.sqrt(1.0 + u @ u), exact


@pytest.mark.parametrize("pusher", [0, 1])
def test_synchrotron_cooling_closed_form(orc, pusher):
    """A particle gyrating perpendicular to a uniform B loses energy at the
    synchrotron rate: with pdot perpendicular to p the bracket of eq:prad is
    gamma^2 pdot^2, which gives gamma' = -kappa (gamma^2 - 1).  The explicit
    scheme converges to that solution at first order in dt."""
    g1, exact = _synchrotron_gamma(orc, 0.05, pusher)
    g2, _ = _synchrotron_gamma(orc, 0.025, pusher)
    e1 = abs(g1 - exact) / (exact - 1.0)
    e2 = abs(g2 - exact) / (exact - 1.0)
    assert exact < 2.1   # gamma fell from 10 to about 2: the cooling dominates the run
    assert e1 < 3e-3 and e2 < 1.5e-3, (e1, e2)
    assert 1.7 < e1 / e2 < 2.3, (e1, e2)


def test_radiated_power_equals_lienard_form_in_three_velocities(orc):
    """eq:prad (proper velocities) is a rewrite of eq:pradv (three-velocities).
    With p- = p0 - pdot dt/2 and p+ = p0 + pdot dt/2 the oracle's p0 and pdot
    are exact, and the energy it removes per step, m (p0 . dp)/(gamma0 dt),
    must equal eq:pradv at v = p0/gamma0, vdot = d(p/gamma)/dt."""
    rng = np.random.default_rng(42)
    K, m, dt = 0.03, 1.0, 0.01
    for _ in range(200):
        g = 1.0 + 10.0 ** rng.uniform(-2, 3)
        p0 = rng.normal(size=3)
        p0 *= math.sqrt(g * g - 1.0) / np.linalg.norm(p0)
        pdot = rng.normal(size=3) * 10.0 ** rng.uniform(-2, 1)
        um, up = p0 - 0.5 * dt * pdot, p0 + 0.5 * dt * pdot
        out = orc.radiate(K, dt, um, up)
        dp = out - up
        gamma0 = math.sqrt(1.0 + p0 @ p0)
        # the change is along -p0 ...
        # (dp is a difference of O(|p|) numbers: tolerances follow |p| eps)
        assert np.linalg.norm(np.cross(dp, p0)) <= 1e-14 * np.linalg.norm(up) * np.linalg.norm(p0)
        assert dp @ p0 < 0.0
        power = -m * (p0 @ dp) / (gamma0 * dt)
        # ... and carries the Lienard power of the three-velocity
        v = p0 / gamma0
        vdot = pdot / gamma0 - p0 * (p0 @ pdot) / gamma0 ** 3
        lienard = K * m * (gamma0 ** 4 * (vdot @ vdot) + gamma0 ** 6 * (vdot @ v) ** 2)
        # eq:pradv itself cancels to relative eps gamma^2 (the paper's reason for eq:prad)
        tol = 1e-13 * np.linalg.norm(up) / np.linalg.norm(dp) + 1e-14 * gamma0 ** 2 + 1e-12
        assert power == pytest.approx(lienard, rel=tol)


def test_radiative_cooling_special_cases(orc):
    u = np.array([0.3, -0.2, 0.5])
    # no acceleration: no radiation; K = 0: no change; p0 = 0: no direction, no change
    assert np.array_equal(orc.radiate(0.1, 0.05, u, u), u)
    assert np.array_equal(orc.radiate(0.0, 0.05, u, 1.1 * u), 1.1 * u)
    assert np.array_equal(orc.radiate(0.1, 0.05, -u, u), u)


def test_cooling_off_leaves_the_step_bit_identical(orc):
    """rad = 0 must not change a single bit of the step (the term is skipped)."""
    from pp_synth import thermal
    L = thermal((8, 8, 8), ppc=4, seed=3)
    sims = []
    for rad in (None, 0.0):
        g = orc.Simulation(L.n, L.d, L.dt, shape_order=3)
        for s in L.species:
            kw = {} if rad is None else {"rad": rad}
            g.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], **kw)
        g.step(2)
        sims.append(g)
    for a in range(3):
        assert np.array_equal(sims[0].E[a], sims[1].E[a])
    assert np.array_equal(sims[0].species[0]["ux"], sims[1].species[0]["ux"])


# --------------------------------------------------------------------------
# 4th-order symplectic step (Sec. III, reading R17)
# --------------------------------------------------------------------------

def _solenoidal_fields(orc, L, seed):
    import pp_synth
    g = orc.make_grid(L.n, L.d, L.dt, field_order=6)
    E, A = pp_synth.random_fields(L.n, seed, 0.05)
    B = [orc.diff(g, A[(a + 2) % 3], (a + 1) % 3, +1) - orc.diff(g, A[(a + 1) % 3], (a + 2) % 3, +1)
         for a in range(3)]
    return E, B


@pytest.mark.parametrize("pusher", [0, 1])
def test_step4_is_time_reversible(orc, pusher):
    """The four substeps form a palindrome (b1 = 0, a1 = a4, a2 = a3, b2 = b4)
    with symmetric kicks, and at alpha = 1/2 the field update is the implicit
    midpoint rule, so three steps of +dt followed by three of -dt return
    particles and fields to round-off.  The plain leap-frog step does not
    (its velocities sit half a step away), which shows the test can tell."""
    import pp_synth
    L = pp_synth.thermal((8, 6, 5), ppc=2, u_th=0.3, dx=0.5, dt=0.25, seed=7)
    E, B = _solenoidal_fields(orc, L, 3)   # eq:EllipticB equals the defining equations for div B = 0
    errs = {}
    for integ in (4, 2):
        sim = orc.Simulation(L.n, L.d, L.dt, shape_order=3, alpha=0.5, pusher=pusher, relax_tol=1e-15,
                             relax_max_iter=3000, integrator=integ)
        for s in L.species:
            sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
        sim.load_fields(E, B)
        E0 = [v.copy() for v in sim.E]
        B0 = [v.copy() for v in sim.B]
        P0 = [{k: s[k].copy() for k in ("x", "y", "z", "ux", "uy", "uz")} for s in sim.species]
        sim.step(3)
        assert max(np.abs(sim.E[a] - E0[a]).max() for a in range(3)) > 0.1   # the state did move
        sim.g.dt = -L.dt
        sim.step(3)
        e = max(max(np.abs(sim.E[a] - E0[a]).max(), np.abs(sim.B[a] - B0[a]).max()) for a in range(3))
        for s, p0 in zip(sim.species, P0):
            for k in ("ux", "uy", "uz"):
                e = max(e, np.abs(s[k] - p0[k]).max())
            for a, k in enumerate("xyz"):
                Lb = L.n[a] * L.d[a]
                e = max(e, np.abs((s[k] - p0[k] + Lb / 2) % Lb - Lb / 2).max())
        errs[integ] = e
    assert errs[4] < 1e-12, errs
    assert errs[2] > 1e-3, errs


def _gyration_error(orc, h, integrator, u0=0.5):
    """Largest position / momentum error of a test particle (weight 1e-10) after
    two gyrations in a uniform B_z = 1 (q = -1, m = 1: u turns counter-clockwise
    at Omega = 1/gamma on a circle of radius u0)."""
    g0 = math.sqrt(1.0 + u0 * u0)
    om = 1.0 / g0
    n = int(round(4.0 * math.pi * g0 / h))
    T = n * h
    sim = orc.Simulation((8, 8, 8), (1.0, 1.0, 1.0), h, shape_order=3, alpha=0.5, relax_tol=1e-14,
                         relax_max_iter=400, integrator=integrator)
    x0 = (3.3, 3.1, 4.2)
    t0 = 0.0 if integrator == 4 else -0.5 * h     # leap-frog velocities lag half a step
    sim.add_species(-1.0, 1.0, 1e-10, [x0[0]], [x0[1]], [x0[2]],
                    [u0 * math.cos(om * t0)], [u0 * math.sin(om * t0)], [0.0])
    E = [np.zeros((8, 8, 8)) for _ in range(3)]
    B = [np.zeros((8, 8, 8)) for _ in range(3)]
    B[2][...] = 1.0
    sim.load_fields(E, B)
    sim.step(n)
    s = sim.species[0]
    xe = x0[0] + u0 * math.sin(om * T)
    ye = x0[1] + u0 * (1.0 - math.cos(om * T))
    tu = T + t0
    dpos = max(abs((s["x"][0] - xe + 4.0) % 8.0 - 4.0), abs((s["y"][0] - ye + 4.0) % 8.0 - 4.0))
    du = max(abs(s["ux"][0] - u0 * math.cos(om * tu)), abs(s["uy"][0] - u0 * math.sin(om * tu)))
    return dpos, du


def test_step4_gyration_converges_at_fourth_order(orc):
    """Against the exact circle, halving dt divides the 4th-order step's error
    by about 16 (the leap-frog's by about 4): the kick sizes cancel the cubic
    phase error of the Vay rotation, 2 w1^3 + w0^3 = 0."""
    e4 = [_gyration_error(orc, h, 4) for h in (0.4, 0.2)]
    e2 = [_gyration_error(orc, h, 2) for h in (0.4, 0.2)]
    for k in range(2):
        assert 13.0 < e4[0][k] / e4[1][k] < 17.0, e4
        assert 3.5 < e2[0][k] / e2[1][k] < 4.5, e2
    assert e4[1][0] < 0.05 * e2[1][0]


@pytest.mark.parametrize("mode", [1, 3])
def test_step4_vacuum_energy_is_product_of_substep_factors(orc, mode):
    """With no particles a 4th-order step is four field updates with dt -> a_i dt:
    the energy of a vacuum mode falls by the product of the theta-scheme's
    closed-form factors (1 + beta^2 s_i^2)/(1 + alpha^2 s_i^2), s_i = a_i dt K(k).
    The a_i are the published drift fractions of the fourth-order composition
    (Forest & Ruth; Candy & Rozmus): w1/2, (w0+w1)/2, (w0+w1)/2, w1/2 with
    w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3) w1."""
    nx, dx, dt, alpha = 16, 0.5, 0.25, 0.55
    sim = orc.Simulation((nx, 2, 2), (dx, dx, dx), dt, field_order=6, alpha=alpha, relax_tol=1e-15,
                         relax_max_iter=500, integrator=4)
    k = 2 * np.pi * mode / (nx * dx)
    kc = orc.fd_coeffs(6)
    K = (2 / dx) * (kc[0] * np.sin(k * dx / 2) + kc[1] * np.sin(3 * k * dx / 2) + kc[2] * np.sin(5 * k * dx / 2))
    w1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    w0 = -(2.0 ** (1.0 / 3.0)) * w1
    ratio = 1.0
    for a in (w1 / 2, (w0 + w1) / 2, (w0 + w1) / 2, w1 / 2):
        s = a * dt * K
        ratio *= (1 + (1 - alpha) ** 2 * s * s) / (1 + alpha ** 2 * s * s)
    x = np.arange(nx) * dx
    E = [np.zeros((2, 2, nx)) for _ in range(3)]
    B = [np.zeros((2, 2, nx)) for _ in range(3)]
    E[1][...] = np.cos(k * x)
    B[2][...] = 0.3 * np.sin(k * (x + dx / 2))
    sim.load_fields(E, B)
    W0 = sum((v ** 2).sum() for v in sim.E + sim.B)
    sim.step(1)
    W1 = sum((v ** 2).sum() for v in sim.E + sim.B)
    assert W1 / W0 == pytest.approx(ratio, rel=1e-12)


# --------------------------------------------------------------------------
# Explicit 6th-order FDTD variant (Sec. VIII cold-beam study, reading R18)
# --------------------------------------------------------------------------

def _K(orc, order, dx, theta):
    kc = orc.fd_coeffs(order)
    return (2 / dx) * (kc[0] * np.sin(theta / 2) + kc[1] * np.sin(3 * theta / 2) + kc[2] * np.sin(5 * theta / 2))


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("mode", [1, 3, 6])
def test_explicit_fdtd_vacuum_dispersion_closed_form(orc, order, mode):
    """A standing vacuum mode E_y ~ cos(kx) under the leap-frog obeys the
    three-term recurrence e(n+1) + e(n-1) = 2 cos(phi) e(n) with the closed-form
    cos(phi) = 1 - (dt K(k))^2 / 2 of the staggered difference symbol K: no
    damping, and the discrete phase speed of the scheme."""
    nx, dx, dt = 16, 0.5, 0.2
    sim = orc.Simulation((nx, 2, 2), (dx, dx, dx), dt, field_order=order, field_solver=orc.EXPLICIT)
    k = 2 * np.pi * mode / (nx * dx)
    x = np.arange(nx) * dx
    E = [np.zeros((2, 2, nx)) for _ in range(3)]
    B = [np.zeros((2, 2, nx)) for _ in range(3)]
    E[1][...] = np.cos(k * x)
    sim.load_fields(E, B)
    basis = np.broadcast_to(np.cos(k * x), (2, 2, nx))
    e = []
    for _ in range(40):
        e.append((sim.E[1] * basis).sum() / (basis * basis).sum())
        sim.step(1)
    e = np.array(e)
    cphi = 1.0 - (dt * _K(orc, order, dx, k * dx)) ** 2 / 2.0
    assert abs(cphi) < 1.0
    assert np.abs(e[2:] + e[:-2] - 2 * cphi * e[1:-1]).max() < 1e-12 * np.abs(e).max()
    assert np.abs(e).max() <= 1.0 + 1e-12 and np.abs(e).max() > 0.5


def test_explicit_fdtd_stability_limit(orc):
    """The leap-frog is stable for dt sqrt(sum_a Kmax_a^2) < 2 and blows up
    just above: random fields (white-noise content reaches the Nyquist mode)
    stay bounded 1% below the limit and grow by orders 1% above it."""
    n, d = (8, 8, 8), (0.5, 0.4, 0.45)
    theta = np.linspace(0, np.pi, 4001)
    kmax2 = sum(np.max(_K(orc, 6, h, theta) ** 2) for h in d)
    dt_c = 2.0 / np.sqrt(kmax2)
    import pp_synth
    E, B = pp_synth.random_fields(n, 5, 1.0)
    W = {}
    for f in (0.99, 1.01):
        sim = orc.Simulation(n, d, f * dt_c, field_order=6, field_solver=orc.EXPLICIT)
        sim.load_fields(E, B)
        W0 = sum((v ** 2).sum() for v in sim.E + sim.B)
        sim.step(150)
        W[f] = sum((v ** 2).sum() for v in sim.E + sim.B) / W0
    assert W[0.99] < 3.0, W
    assert W[1.01] > 1e6, W


@pytest.mark.parametrize("shape", [2, 3])
def test_explicit_fdtd_keeps_gauss_and_divB_with_particles(orc, shape):
    """With the charge-conserving current the explicit update keeps div^- E - rho
    and div^+ B at their initial values (curl and divergence commute on the
    staggered mesh), like the implicit one."""
    import pp_synth
    L = pp_synth.thermal(n=(8, 6, 5), ppc=2, u_th=0.3, dx=0.5, dt=0.1, seed=7)
    sim = orc.Simulation(L.n, L.d, L.dt, field_order=6, shape_order=shape, field_solver=orc.EXPLICIT)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    E, B = _solenoidal_fields(orc, L, 4)
    sim.load_fields(E, B)
    g0 = orc.div_minus(sim.g, sim.E) - sim.rho()
    b0 = orc.div_plus(sim.g, sim.B)
    moved = 0.0
    for _ in range(6):
        sim.step(1)
        moved = max(moved, np.abs(orc.div_minus(sim.g, sim.E) - g0).max())
        assert np.abs(orc.div_minus(sim.g, sim.E) - sim.rho() - g0).max() < 1e-12 * max(1.0, np.abs(g0).max())
        assert np.abs(orc.div_plus(sim.g, sim.B) - b0).max() < 1e-12
    assert moved > 1e-4     # the charge did move


# --------------------------------------------------------------------------
# Direct current eq:jj2 (reading R19) and the divergence filter (reading R20)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [1, 2, 3])
def test_direct_current_moments(orc, shape):
    """With J = sum q w v W(x_mid - x_c) on the staggered nodes, the total of
    each component is sum q w v_a (partition of unity) and its first moment
    along every axis is sum q w v_a x_mid (B-splines of order >= 1 reproduce
    linear functions).  Particles stay clear of the periodic seam."""
    n, d, dt = (12, 10, 11), (0.5, 0.4, 0.45), 0.2
    rng = np.random.default_rng(shape)
    m = 400
    x0 = [rng.uniform(3.5, n[a] - 3.5, m) * d[a] for a in range(3)]
    u = [rng.normal(0, 0.4, m) for _ in range(3)]
    sim = orc.Simulation(n, d, dt, shape_order=shape, current_mode=orc.DIRECT)
    sim.add_species(-1.0, 1.0, 0.3, x0[0], x0[1], x0[2], u[0], u[1], u[2])
    sim.deposit()   # E = B = 0: the momenta do not change
    g = np.sqrt(1 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    v = [u[a] / g for a in range(3)]
    xm = [x0[a] + 0.5 * dt * v[a] for a in range(3)]
    qw = -0.3
    nz, ny, nx = n[2], n[1], n[0]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for a in range(3):
        J = sim.J[a]
        assert J.sum() == pytest.approx(qw * v[a].sum(), rel=1e-12)
        for b, idx in enumerate((i, j, k)):
            xn = (idx + (0.5 if b == a else 0.0)) * d[b]     # J_a sits half a cell up along a
            assert (J * xn).sum() == pytest.approx((qw * v[a] * xm[b]).sum(), rel=1e-11, abs=1e-12)


def test_direct_current_breaks_gauss_law_charge_conserving_keeps_it(orc):
    """The reason the paper replaced eq:jj2: with it div^- E - rho drifts from
    its initial value; with the charge-conserving current it stays put."""
    import pp_synth
    L = pp_synth.thermal(n=(8, 6, 5), ppc=2, u_th=0.3, dx=0.5, dt=0.25, seed=7)
    drift = {}
    for mode in (orc.CHARGE_CONSERVING, orc.DIRECT):
        sim = orc.Simulation(L.n, L.d, L.dt, shape_order=2, current_mode=mode)
        for s in L.species:
            sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
        g0 = orc.div_minus(sim.g, sim.E) - sim.rho()
        sim.step(3)
        drift[mode] = np.abs(orc.div_minus(sim.g, sim.E) - sim.rho() - g0).max() / np.abs(sim.rho()).max()
    assert drift[orc.CHARGE_CONSERVING] < 1e-12
    assert drift[orc.DIRECT] > 1e-4


def test_divergence_filter_removes_nyquist_error_in_one_pass(orc):
    """tau = 1/max(sum K^2): the checkerboard error is the eigenmode of the
    largest eigenvalue of -div grad, so one pass removes it from E and B."""
    n, d = (8, 8, 8), (0.5, 0.4, 0.45)
    sim = orc.Simulation(n, d, 0.1, field_order=6)
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    cb = (-1.0) ** (i + j + k)
    # E with div^- E = checkerboard and rho = 0; B with div^+ B = checkerboard
    g = sim.g
    E = [np.zeros((8, 8, 8)) for _ in range(3)]
    E[0] = cb.copy()
    B = [np.zeros((8, 8, 8)) for _ in range(3)]
    B[2] = cb.copy()
    sim.load_fields(E, B)
    e0 = np.abs(orc.div_minus(g, sim.E)).max()
    b0 = np.abs(orc.div_plus(g, sim.B)).max()
    sim.divergence_filter(1)
    assert e0 > 1.0 and b0 > 1.0
    assert np.abs(orc.div_minus(g, sim.E)).max() < 1e-12 * e0
    assert np.abs(orc.div_plus(g, sim.B)).max() < 1e-12 * b0


def test_divergence_filter_converges_by_gradients_only(orc):
    """Many passes drive div^- E - rho to its (unremovable) mean and div^+ B to
    zero, and change E and B by discrete gradients only: the curls of the
    changes vanish, so the filter leaves the induction equations alone."""
    import pp_synth
    n, d = (6, 6, 6), (0.5, 0.5, 0.5)
    L = pp_synth.thermal(n=n, ppc=2, u_th=0.3, dx=0.5, dt=0.1, seed=3)
    sim = orc.Simulation(n, d, 0.1, field_order=6)
    sim.add_species(L.species[0]["q"], 1.0, L.species[0]["w"], *(L.species[0][k] for k in ("x", "y", "z", "ux", "uy", "uz")))
    E, B = pp_synth.random_fields(n, 2, 1.0)
    sim.load_fields(E, B)
    E0 = [v.copy() for v in sim.E]
    B0 = [v.copy() for v in sim.B]
    g = sim.g
    rho = sim.rho()
    e_start = orc.div_minus(g, sim.E) - rho
    sim.divergence_filter(600)
    e = orc.div_minus(g, sim.E) - rho
    assert np.abs(e - e.mean()).max() < 1e-10 * np.abs(e_start).max()
    assert e.mean() == pytest.approx(e_start.mean(), abs=1e-12)
    assert np.abs(orc.div_plus(g, sim.B)).max() < 1e-10 * np.abs(orc.div_plus(g, B0)).max()
    def curl(F, sign):
        out = []
        for a in range(3):
            b, c = (a + 1) % 3, (a + 2) % 3
            out.append(orc.diff(g, F[c], b, sign) - orc.diff(g, F[b], c, sign))
        return out
    dE = [sim.E[a] - E0[a] for a in range(3)]
    dB = [sim.B[a] - B0[a] for a in range(3)]
    assert max(np.abs(c).max() for c in curl(dE, +1)) < 1e-12 * max(np.abs(x).max() for x in dE)
    assert max(np.abs(c).max() for c in curl(dB, -1)) < 1e-12 * max(np.abs(x).max() for x in dB)


def test_threaded_particle_loop_equals_the_plain_one(orc):
    """The oracle's particle loop on several threads (per-thread copies of the
    charge change and line sums, added after the loop: the timing baseline's
    all-core form) gives the single-threaded results to summation order
    (1e-13), for the charge-conserving and the direct current."""
    import pp_synth
    from tests import gpu_helpers as H
    L = pp_synth.thermal(n=(8, 8, 8), ppc=8, u_th=0.1, dx=0.1, dt=0.05, seed=5)
    for mode in (orc.CHARGE_CONSERVING, orc.DIRECT):
        runs = []
        for nt in (1, 4):
            orc.set_threads(nt)
            sim = orc.Simulation(L.n, L.d, L.dt, shape_order=3, relax_tol=1e-14, relax_max_iter=2000,
                                 current_mode=mode)
            for s in L.species:
                sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
            sim.step(2)
            runs.append(sim)
        orc.set_threads(1)
        for F in ("E", "B", "J"):
            a, b = getattr(runs[0], F), getattr(runs[1], F)
            scale = max(np.abs(x).max() for x in a)
            assert max(np.abs(x - y).max() for x, y in zip(a, b)) <= 1e-13 * scale, (mode, F)
        for s in range(2):   # the second step's push sees fields that differ at round-off
            for k in ("x", "ux"):
                a, b = runs[0].species[s][k], runs[1].species[s][k]
                assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max(), (mode, s, k)


@pytest.mark.slow
def test_quiet_filamentation_growth_matches_cold_fluid_theory(orc):
    """The oracle's quiet-start filamentation (Weibel) instability of cold
    counter-streaming pair beams (+-0.5c along x, density 1/2 per population)
    with one seeded transverse mode grows at the rate of the cold-fluid
    dispersion relation within 5% (the discrete scheme and the shape factor
    shift it slightly at k dy = 0.39)."""
    import pp_synth
    from tests import theory
    L = pp_synth.quiet_weibel()
    sim = orc.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=2, relax_tol=1e-13,
                         relax_max_iter=2000)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    W = []
    for _ in range(240):
        sim.step(1)
        W.append(sim.diagnostics()["energy_B"])
    t = np.arange(1, 241) * L.dt
    rate, npts = theory.fit_growth(t, np.array(W))
    assert npts >= 30
    expect = theory.cold_filamentation(L.params["k"], [(0.5, 0.5)] * 4)
    assert rate == pytest.approx(expect, rel=0.05), (rate, expect)
