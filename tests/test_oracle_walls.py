"""Pins of the oracle's reflecting walls (Sec. II "Boundary conditions").

The oracle builds the wall from its definition, virtual mirror images in the
mirror-extended periodic box.  These tests hold that construction to things
outside it: the closed-form path of a free particle between two mirrors, the
mirror symmetry that the Maxwell equations and the paper's parity table
imply (which a wrong parity, a wrong image momentum or a wrong mirror index
breaks within a step), exact charge conservation, and the paper's own
folding rules for rho, J_par and J_perp, which must reproduce the images'
deposit.
"""

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
