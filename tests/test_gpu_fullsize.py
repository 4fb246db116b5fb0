"""Parity at the benchmark's full size and launch configuration: 128^3 cells,
32 macro-particles per cell per species (134,217,728 particles), PCS, 6th-order
fields, mixed precision, tiled deposit.

The oracle cannot run the whole box, so it checks what it can compute one by
one -- sampled particles followed through a step (between cell sorts the
library keeps the particle order): gather from the GPU's own fields, Vay push
and move, in FP64 -- and properties that hold at any size: the total current
equals sum q w v, the total charge stays zero, and Gauss's law drifts only at
FP32 round-off.
"""
import numpy as np
import pytest

import pp_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as pp
    L = pp_synth.thermal()                     # 128^3 x 32 ppc x 2 species, seed 1212
    sim = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3, pusher=pp.PP_VAY,
                        precision=pp.PP_MIXED32, sort_interval=20, relax_max_iter=100, relax_tol=1e-6,
                        deposit_mode=pp.PP_DEPOSIT_TILED)
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]))
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    return pp, L, sim


def test_fullsize_sampled_particles_match_oracle(full, orc):
    pp, L, sim = full
    sim.step(2)                                # fields become nonzero after the first step
    E, B, _ = sim.fields()
    before = sim.particles(0)
    rng = np.random.default_rng(5)
    idx = rng.choice(len(before["x"]), size=2000, replace=False)
    sim.step(1)
    after = sim.particles(0)
    d = sim.diagnostics()
    assert d["status"] == 0
    g = orc.make_grid(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3)
    q, m = L.species[0]["q"], L.species[0]["m"]
    box = np.array([L.n[a] * L.d[a] for a in range(3)])
    worst_x = worst_u = 0.0
    for i in idx:
        x0 = np.array([before["x"][i], before["y"][i], before["z"][i]])
        u0 = np.array([before["ux"][i], before["uy"][i], before["uz"][i]])
        Ep, Bp = orc.gather(g, E, B, x0)
        u1 = orc.push(q * L.dt / m, Ep, Bp, u0)
        x1 = x0 + L.dt * u1 / np.sqrt(1.0 + u1 @ u1)
        got_x = np.array([after["x"][i], after["y"][i], after["z"][i]])
        got_u = np.array([after["ux"][i], after["uy"][i], after["uz"][i]])
        dx = (got_x - x1 + 0.5 * box) % box - 0.5 * box
        worst_x = max(worst_x, np.abs(dx).max())
        worst_u = max(worst_u, np.abs(got_u - u1).max() / max(np.abs(u1).max(), 1e-3))
    # FP32 offsets of a 0.1-wide cell (~1e-8) and FP32 momenta and gathered fields
    assert worst_x <= 2e-6, worst_x
    assert worst_u <= 2e-5, worst_u


def test_fullsize_current_charge_and_gauss(full):
    pp, L, sim = full
    sim.step(1)
    sim.deposit(-1)            # the particle half only: J of this half step stays on the mesh
    _, _, J = sim.fields()
    after = [sim.particles(s) for s in range(2)]
    # sum of J over the mesh = sum over particles of q w v^{n+1/2} (B-spline linear
    # reproduction; the high-order solve keeps every line mean)
    for a, k in enumerate(("ux", "uy", "uz")):
        expect = 0.0
        mag = 0.0
        for s, sp in enumerate(L.species):
            P = after[s]
            v = P[k] / np.sqrt(1.0 + P["ux"] ** 2 + P["uy"] ** 2 + P["uz"] ** 2)
            expect += sp["q"] * sp["w"] * float(np.sum(v))
            mag += abs(sp["q"] * sp["w"]) * float(np.sum(np.abs(v)))
        assert abs(J[a].sum() - expect) <= 1e-5 * mag, (a, J[a].sum(), expect, mag)
    sim.field_update()
    d = sim.diagnostics()
    assert d["status"] == 0
    assert abs(d["charge"]) <= 1e-6 * d["n_particles"] * L.species[0]["w"] * np.prod(L.d)
    assert d["gauss_drift_max"] <= 2e-5 * d["rho_max"]
    assert d["n_slow"] >= 0
