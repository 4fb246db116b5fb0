"""Pins of the oracle's reflecting walls (Sec. V "Boundary conditions").

The oracle builds the wall from its definition, virtual mirror images in the
mirror-extended periodic box.  These tests hold that construction to things
outside it: the closed-form path of a free particle between two mirrors, the
mirror symmetry that the Maxwell equations and the paper's parity table
imply (which a wrong parity, a wrong image momentum or a wrong mirror index
breaks within a step), exact charge conservation, and the paper's own
folding rules for rho, J_par and J_perp, which must reproduce the images'
deposit.
"""

import math
import os

import numpy as np
import pytest

import pp_synth


def _fold(F, half, sign):
    """The paper's folding of a deposit made by the particles alone:
    f(x_b - dx) += P f(x_b + dx), written for the whole extended box."""
    import oracle
    return F + oracle.mirror_x(F, half, sign)


def test_free_particle_bounces_between_walls(orc):
    """Two light particles (weight 1e-13: their own field is negligible) in
    empty fields, one heading for each wall: after k steps each sits at the
    folded position of the straight path x0 + k dt v_x (triangle wave of
    period 2L) with u_x reversed on the odd legs, and y, z move freely."""
    n, d, dt = (16, 8, 8), (0.5, 0.5, 0.5), 0.2
    L = n[0] * d[0]
    x0 = np.array([6.7, 1.1])
    u0 = np.array([[2.0, 0.3, -0.1], [-1.5, -0.2, 0.4]])
    sim = orc.WallSimulation(n, d, dt, shape_order=3)
    sim.add_species(-1.0, 1.0, 1e-13, x0, np.array([1.3, 2.2]), np.array([0.7, 3.1]),
                    u0[:, 0], u0[:, 1], u0[:, 2])
    g = np.sqrt(1.0 + (u0 ** 2).sum(1))
    v = u0 / g[:, None]
    for k in range(10, 101, 10):
        sim.step(10)
        p = sim.particles(0)
        X = x0 + k * dt * v[:, 0]
        s = np.mod(X, 2 * L)
        xe = np.where(s <= L, s, 2 * L - s)
        uxe = np.where(s <= L, u0[:, 0], -u0[:, 0])
        assert np.abs(p["x"] - xe).max() < 1e-9, (k, p["x"], xe)
        assert np.abs(p["ux"] - uxe).max() < 1e-9, (k, p["ux"], uxe)
        ye = np.mod(np.array([1.3, 2.2]) + k * dt * v[:, 1], n[1] * d[1])
        assert np.abs(p["y"] - ye).max() < 1e-9
        assert np.abs(p["uy"] - u0[:, 1]).max() < 1e-9 and np.abs(p["uz"] - u0[:, 2]).max() < 1e-9
    # the path crossed both walls
    assert (x0[0] + 100 * dt * v[0, 0]) > 2 * L and (x0[1] + 100 * dt * v[1, 0]) < 0.0


def _random_wall_sim(orc, shape=3, steps=3, solver=None, seed=41):
    n, d, dt = (12, 6, 6), (0.5, 0.45, 0.4), 0.2
    L = pp_synth.random_particles(n, d, dt, 800, seed=seed, u_scale=0.5)
    kw = {} if solver is None else dict(field_solver=solver)
    sim = orc.WallSimulation(n, d, L.dt if solver is None else 0.1, shape_order=shape, **kw)
    s = L.species[0]
    sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    E, B = pp_synth.random_fields((2 * n[0], n[1], n[2]), seed + 1, 0.05)
    sim.load_fields(E, B)
    sim.step(steps)
    return sim, n, d


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_mirror_symmetry_is_kept(orc, shape):
    """Random particles and fields, three steps: every field and current
    component of the extended box keeps the parity of the table (to round-off),
    and each image is still the mirror of its particle."""
    sim, n, d = _random_wall_sim(orc, shape)
    for kind, F in (("E", sim.E), ("B", sim.B), ("J", sim.J)):
        for a in range(3):
            half, sign = orc.WALL_PARITY[kind][a]
            err = np.abs(F[a] - orc.mirror_x(F[a], half, sign)).max()
            assert err <= 1e-12 * np.abs(F[a]).max(), (kind, a, err)
    s = sim.sim.species[0]
    m = sim.counts[0]
    L2 = 2 * n[0] * d[0]
    dx = (s["x"][:m] + s["x"][m:]) % L2
    dx = np.minimum(dx, L2 - dx)
    assert dx.max() < 1e-12
    assert np.abs(s["ux"][:m] + s["ux"][m:]).max() < 1e-12
    for k in ("y", "z", "uy", "uz"):
        assert np.abs(s[k][:m] - s[k][m:]).max() < 1e-12


def test_a_wrong_parity_breaks_the_symmetry(orc):
    """The symmetry check above has teeth: with B_x made odd instead of even
    the evolved state leaves the (wrong) symmetric subspace at once."""
    n, d, dt = (12, 6, 6), (0.5, 0.45, 0.4), 0.2
    sim = orc.Simulation((2 * n[0], n[1], n[2]), d, dt, shape_order=2)
    E, B = pp_synth.random_fields((2 * n[0], n[1], n[2]), 5, 0.05)
    E = orc.wall_symmetrise(E, "E")
    B = [0.5 * (B[a] + orc.mirror_x(B[a], orc.WALL_PARITY["B"][a][0], -orc.WALL_PARITY["B"][a][1]))
         for a in range(3)]
    sim.load_fields(E, B)
    sim.step(1)
    bad = max(np.abs(sim.B[a] - orc.mirror_x(sim.B[a], orc.WALL_PARITY["B"][a][0], -orc.WALL_PARITY["B"][a][1])).max()
              for a in range(3))
    assert bad > 1e-4


def test_charge_is_conserved_between_walls(orc):
    sim, n, d = _random_wall_sim(orc, 3, steps=0)
    d0 = sim.diagnostics()
    # rho = q w sum W per particle (weights sum to one), so sum rho dV = q w N dV
    q = sim.sim.species[0]["q"] * sim.sim.species[0]["w"] * sim.counts[0] * d[0] * d[1] * d[2]
    assert d0["charge"] == pytest.approx(q, rel=1e-12)
    rho0 = sim.rho()
    g0 = orc.div_minus(sim.g, sim.E) - rho0
    sim.step(4)
    d1 = sim.diagnostics()
    assert d1["charge"] == pytest.approx(q, rel=1e-12)
    g1 = orc.div_minus(sim.g, sim.E) - sim.rho()
    assert np.abs(g1 - g0).max() <= 1e-11 * np.abs(rho0).max()


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_paper_folding_rules_reproduce_the_images(orc, shape):
    """rho(x_b - dx) += rho(x_b + dx), J_par likewise, J_perp with a minus
    sign: the particles' own deposit on the extended box, folded by those
    rules, equals the deposit of particles plus images (one step's current,
    and the charge density)."""
    n, d, dt = (12, 6, 6), (0.5, 0.45, 0.4), 0.2
    L = pp_synth.random_particles(n, d, dt, 500, seed=77 + shape, u_scale=0.6)
    s = L.species[0]
    walls = orc.WallSimulation(n, d, dt, shape_order=shape)
    walls.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    alone = orc.Simulation((2 * n[0], n[1], n[2]), d, dt, shape_order=shape)
    alone.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    rho = walls.rho()
    rf = _fold(alone.rho(), False, 1.0)
    assert np.abs(rf - rho).max() <= 1e-13 * np.abs(rho).max()
    walls.sim.deposit()
    alone.deposit()
    for a in range(3):
        half, sign = orc.WALL_PARITY["J"][a]
        jf = _fold(alone.J[a], half, sign)
        assert np.abs(jf - walls.J[a]).max() <= 1e-12 * np.abs(walls.J[a]).max(), a


# --------------------------------------------------------------------------
# Open lower end, injector and sliding window (readings R22-R24)
# --------------------------------------------------------------------------

def test_philox_known_answers(orc):
    """orc_philox4x32 against the published known-answer vectors of
    Philox4x32-10 (tests/golden/philox4x32_10_kat.txt): the all-zero, the
    all-ones and the pi-digits counter/key.  A swapped multiplier, Weyl
    constant, output word or round count fails at least one of them."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert list(orc.philox4x32(v[0:4], v[4:6])) == v[6:10], r
    # orc_draws: draw i is the generator at counter (i, 0, step, stream) under
    # key (seed low, seed high), each word r mapped to (r + 1/2) 2^-32
    seed, step, stream = (0x299f31d0 << 32) | 0xa4093822, 0x13198a2e, 0x03707344
    D = orc.draws(seed, step, stream, 3)
    for i in range(3):
        words = orc.philox4x32((i, 0, step, stream), (0xa4093822, 0x299f31d0))
        assert list(D[i]) == [(w + 0.5) * 2.0 ** -32 for w in words]


def test_philox_draws_are_uniform_and_mix(orc):
    """The counter-based generator of the injector: its words are uniform
    (chi-square over 16 bins), its Box-Muller normals have mean 0 and variance
    1, and one flipped counter or key bit changes about half of the 128 output
    bits (avalanche), for every word of the counter."""
    D = orc.draws(12345, 7, 3, 20000)
    assert D.min() > 0.0 and D.max() < 1.0
    for m in range(4):
        h, _ = np.histogram(D[:, m], bins=16, range=(0.0, 1.0))
        chi2 = ((h - 1250.0) ** 2 / 1250.0).sum()
        assert chi2 < 45.0, (m, chi2)   # 15 degrees of freedom: p ~ 1e-4
    G = orc.gaussians(D)
    assert np.abs(G.mean(0)).max() < 0.03 and np.abs(G.var(0) - 1.0).max() < 0.05
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2)]
        a = orc.philox4x32(ctr, key)
        w, b = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        if w < 4:
            ctr[w] ^= 1 << b
        else:
            key[w - 4] ^= 1 << b
        c = orc.philox4x32(ctr, key)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, c)))
    assert 60.0 < np.mean(flips) < 68.0 and min(flips) > 35


def _inject_sim(orc, n=(16, 4, 4), ppc=3.0, u=(1.2, 0.0, 0.0), u_th=0.0, w=1e-12, seeds=(9, 9)):
    d, dt = (0.5, 0.5, 0.5), 0.2
    sim = orc.WallSimulation(n, d, dt, shape_order=2)
    e = np.zeros(0)
    for q, s in zip((-1.0, 1.0), seeds):
        sid = sim.add_species(q, 1.0, w, e, e, e, e, e, e)
        sim.set_injector(sid, ppc, u, u_th, s)
    return sim, n, d, dt


def test_injector_counts_and_free_streaming_slab(orc):
    """A cold light beam injected for k steps: exactly floor(k r) particles,
    r = ppc ny nz v dt / dx; each batch sits where free streaming puts it (the
    whole inflow fills [0, k v dt) uniformly, no particle outside it), every
    momentum is the drift, and two species with one seed land on the same
    points (a neutral inflow)."""
    sim, n, d, dt = _inject_sim(orc)
    u = 1.2
    v = u / math.sqrt(1 + u * u)
    r = 3.0 * n[1] * n[2] * v * dt / d[0]
    for k in range(1, 21):
        sim.step(1)
        p0, p1 = sim.particles(0), sim.particles(1)
        assert len(p0["x"]) == len(p1["x"]) == math.floor(k * r)
    p0, p1 = sim.particles(0), sim.particles(1)
    assert np.abs(p0["ux"] - u).max() < 1e-9 and np.abs(p0["uy"]).max() < 1e-9
    assert p0["x"].min() > 0.0 and p0["x"].max() < 20 * v * dt + 1e-9
    # uniform fill: the count below every depth is proportional to it
    for depth in (0.25, 0.5, 0.75):
        frac = (p0["x"] < depth * 20 * v * dt).mean()
        assert abs(frac - depth) < 0.05, (depth, frac)
    o0 = np.lexsort((p0["z"], p0["y"], p0["x"]))
    o1 = np.lexsort((p1["z"], p1["y"], p1["x"]))
    for k in ("x", "y", "z"):
        assert np.abs(p0[k][o0] - p1[k][o1]).max() < 1e-9
    dg = sim.diagnostics()
    assert abs(dg["charge"]) < 1e-20


def test_open_layer_absorbs_an_outgoing_wave(orc):
    """A transverse vacuum pulse (E_y, B_z) running towards x = 0: with a
    20-cell layer most of its energy is gone once it has been and come back;
    with the bare mirror (no layer) the energy stays."""
    n, d, dt = (48, 4, 4), (0.5, 0.5, 0.5), 0.1
    out = {}
    for layer in (False, True):
        sim = orc.WallSimulation(n, d, dt, shape_order=1, field_solver=orc.EXPLICIT)
        N = 2 * n[0]
        xi = np.arange(N, dtype=float)
        xh = xi + 0.5
        pulse = lambda x: np.exp(-((x - 30.0) / 3.0) ** 2) * (x < n[0])
        E = [np.zeros((n[2], n[1], N)) for _ in range(3)]
        B = [np.zeros((n[2], n[1], N)) for _ in range(3)]
        E[1][...] = pulse(xi)
        B[2][...] = -pulse(xh)          # E x B along -x
        sim.load_fields(E, B)
        if layer:
            sim.set_open_boundary(20, 0.3, 0.0)
        e0 = sim.diagnostics()
        sim.step(int(round(2 * 30 * d[0] / dt)) + 40)
        e1 = sim.diagnostics()
        out[layer] = (e1["energy_E"] + e1["energy_B"]) / (e0["energy_E"] + e0["energy_B"])
    assert out[False] > 0.95 and out[True] < 0.1, out


def test_escape_takes_outgoing_particles_only(orc):
    """Light particles in empty fields near the open end: those moving out
    leave at the first step that ends below `escape` cells; those moving in,
    and everything while no open end is set, stay."""
    n, d, dt = (16, 4, 4), (0.5, 0.5, 0.5), 0.2
    sim = orc.WallSimulation(n, d, dt, shape_order=2)
    x0 = np.array([2.0, 2.0, 3.0])
    ux = np.array([-1.0, 1.0, -0.5])
    o = np.array([1.0, 1.0, 1.0])
    sim.add_species(-1.0, 1.0, 1e-12, x0, o, o, ux, 0 * o, 0 * o)
    sim.set_open_boundary(8, 0.0, 3.0)
    v = ux / np.sqrt(1 + ux * ux)
    for k in range(1, 25):
        sim.step(1)
        x = x0 + k * dt * v
        alive = ~((x < 3.0 * d[0]) & (v < 0))
        # a particle once gone stays gone
        if k > 1:
            alive &= prev
        assert len(sim.particles(0)["x"]) == alive.sum(), k
        prev = alive
    assert alive.tolist() == [False, True, False]


def test_window_shifts_content_and_adds_a_layer(orc):
    """Window at v = 0.6: shifts happen exactly when floor(k v dt / dx) grows;
    at a shift the fields equal those of an identical run without the window
    moved up one cell (zero in the new bottom layer), particles moved up by
    dx, the top layer's particles gone, and a new layer of round(ppc ny nz)
    injected particles in [0, dx)."""
    n, d, dt = (12, 4, 4), (0.5, 0.5, 0.5), 0.2
    L = pp_synth.random_particles(n, d, dt, 300, seed=5, u_scale=0.2)
    s = L.species[0]
    runs = []
    for window in (False, True):
        sim = orc.WallSimulation(n, d, dt, shape_order=2)
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
        sid = sim.add_species(1.0, 1.0, 0.05, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0),
                              np.zeros(0))
        sim.injectors[sid] = dict(ppc=2.0, u=np.array([0.3, 0.0, 0.0]), u_th=0.1, seed=4, k0=0)
        E, B = pp_synth.random_fields((2 * n[0], n[1], n[2]), 6, 0.05)
        sim.load_fields(E, B)
        if window:
            sim.set_window(0.6)
        runs.append(sim)
    plain, win = runs
    frac = 0.6 * dt / d[0]
    shifts = 0
    for k in range(1, 12):
        plain.step(1)
        win.step(1)
        if math.floor(k * frac) > math.floor((k - 1) * frac):
            shifts += 1
            assert win.shifts == shifts
            # fields: the plain run's, one cell up (physical half), zero at the bottom
            assert np.abs(win.sim.E[1][..., 1:n[0] + 1] - plain.sim.E[1][..., 0:n[0]]).max() < 1e-12
            assert np.abs(win.sim.E[1][..., 0]).max() == 0.0
            assert np.abs(win.sim.E[0][..., 1:n[0]] - plain.sim.E[0][..., 0:n[0] - 1]).max() < 1e-12
            # the new layer
            p1 = win.particles(1)
            fresh = p1["x"] < d[0]
            assert fresh.sum() >= round(2.0 * n[1] * n[2])
            break
    assert shifts == 1
    # after the shift the window run's particles are the plain run's moved up by dx
    pw, pp_ = win.particles(0), plain.particles(0)
    xs = np.sort(pp_["x"] + d[0])
    xs = xs[xs <= n[0] * d[0]]
    assert np.abs(np.sort(pw["x"]) - xs).max() < 1e-12


# --------------------------------------------------------------------------
# Walls on y and z (and on several axes at once)
# --------------------------------------------------------------------------

def test_wall_parity_table_for_every_normal(orc):
    """The generic table reduces to the paper's for the x normal, and for any
    normal a the staggered components (E_a, J_a; B_b for b != a) are odd."""
    for kind in ("E", "B", "J"):
        for comp in range(3):
            assert orc.wall_parity(kind, comp, 0) == orc.WALL_PARITY[kind][comp]
    assert orc.wall_parity("E", 1, 1) == (True, -1.0) and orc.wall_parity("B", 1, 1) == (False, 1.0)
    assert orc.wall_parity("B", 0, 2) == (True, -1.0) and orc.wall_parity("J", 0, 2) == (False, 1.0)


def test_free_particle_bounces_in_a_closed_box(orc):
    """Walls on all three axes: each coordinate of a light particle in empty
    fields follows its own folded straight path, with that velocity component
    reversed on its odd legs."""
    n, d, dt = (8, 6, 4), (0.5, 0.5, 0.5), 0.2
    Ls = np.array([n[a] * d[a] for a in range(3)])
    x0 = np.array([[2.7, 1.1, 0.6], [0.3, 2.2, 1.7]])
    u0 = np.array([[1.5, -0.9, 0.7], [-0.4, 1.2, -1.1]])
    sim = orc.WallSimulation(n, d, dt, walls=(True, True, True), shape_order=2)
    sim.add_species(-1.0, 1.0, 1e-13, x0[:, 0], x0[:, 1], x0[:, 2], u0[:, 0], u0[:, 1], u0[:, 2])
    v = u0 / np.sqrt(1.0 + (u0 ** 2).sum(1))[:, None]
    for k in (10, 25, 40):
        sim.step(k - sim.nstep)
        p = sim.particles(0)
        for a in range(3):
            s = np.mod(x0[:, a] + k * dt * v[:, a], 2 * Ls[a])
            xe = np.where(s <= Ls[a], s, 2 * Ls[a] - s)
            ue = np.where(s <= Ls[a], u0[:, a], -u0[:, a])
            assert np.abs(p["xyz"[a]] - xe).max() < 1e-9, (k, a)
            assert np.abs(p["u" + "xyz"[a]] - ue).max() < 1e-9, (k, a)


@pytest.mark.parametrize("walls", [(False, True, False), (False, False, True), (True, True, True)])
def test_mirror_symmetry_kept_for_other_walls(orc, walls):
    """Random particles and fields between walls on y, on z, or on all three
    axes, three steps: every component keeps the parity of its wall normal
    across every walled axis (to round-off)."""
    n, d, dt = (8, 6, 6), (0.5, 0.45, 0.4), 0.2
    L = pp_synth.random_particles(n, d, dt, 300, seed=61, u_scale=0.5)
    s = L.species[0]
    sim = orc.WallSimulation(n, d, dt, walls=walls, shape_order=3)
    sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    ext = tuple(2 * n[a] if walls[a] else n[a] for a in range(3))
    E, B = pp_synth.random_fields(ext, 62, 0.05)
    sim.load_fields(E, B)
    sim.step(3)
    for kind, F in (("E", sim.E), ("B", sim.B), ("J", sim.J)):
        for ax in range(3):
            if not walls[ax]:
                continue
            for c in range(3):
                err = np.abs(F[c] - orc.mirror(F[c], ax, *orc.wall_parity(kind, c, ax))).max()
                assert err <= 1e-12 * max(np.abs(F[c]).max(), 1e-300), (kind, c, ax, err)
    q = s["q"] * s["w"] * len(s["x"]) * d[0] * d[1] * d[2]
    assert sim.diagnostics()["charge"] == pytest.approx(q, rel=1e-12)


def test_folding_rules_on_y(orc):
    """The paper's folding rules with the y normal (rho, J_x, J_z added across
    the wall, J_y subtracted) reproduce the images' deposit."""
    n, d, dt = (6, 8, 6), (0.5, 0.45, 0.4), 0.2
    L = pp_synth.random_particles(n, d, dt, 400, seed=63, u_scale=0.6)
    s = L.species[0]
    walls = orc.WallSimulation(n, d, dt, walls=(False, True, False), shape_order=3)
    walls.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    alone = orc.Simulation((n[0], 2 * n[1], n[2]), d, dt, shape_order=3)
    alone.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    rho = walls.rho()
    assert np.abs(alone.rho() + orc.mirror(alone.rho(), 1, False, 1.0) - rho).max() <= 1e-13 * np.abs(rho).max()
    walls.sim.deposit()
    alone.deposit()
    for c in range(3):
        jf = alone.J[c] + orc.mirror(alone.J[c], 1, *orc.wall_parity("J", c, 1))
        assert np.abs(jf - walls.J[c]).max() <= 1e-12 * np.abs(walls.J[c]).max(), c
