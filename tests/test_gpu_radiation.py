"""GPU parity of radiative cooling (Sec. "Radiative cooling", eq:prad, eq:udot)
through pp_set_radiative_cooling, against the FP64 oracle and the synchrotron
closed form."""
import math

import numpy as np
import pytest

import pp_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4575_gb300 as m
    from paper_1211_4575_gb300 import build
    build.build()
    return m


def _uniform_B(n, Bz):
    nx, ny, nz = n
    E = [np.zeros((nz, ny, nx)) for _ in range(3)]
    B = [np.zeros((nz, ny, nx)) for _ in range(3)]
    B[2][...] = Bz
    return E, B


@pytest.mark.parametrize("precision,mode,tol", [(0, 0, 1e-9), (1, 1, 1e-4), (1, 2, 1e-4)])
def test_synchrotron_single_particle(pp, orc, precision, mode, tol):
    """One particle (gamma 10, weight 1e-12: no self-field to speak of) gyrating
    in a uniform B_z = 1 for 180 steps with K = 0.01: gamma falls to about 2.
    The GPU follows the oracle's push + cooling loop (FP64 to 1e-9, mixed to
    1e-4) and the closed form (gamma-1)/(gamma+1) ~ exp(-2 K (q/m)^2 B^2 t)
    to the scheme's first-order error (0.74% at this dt)."""
    n, d, dt, K, g0, nsteps = (16, 16, 16), (0.5, 0.5, 0.5), 0.25, 0.01, 10.0, 180
    sim = pp.Simulation(n, d, dt, shape_order=3, precision=precision, deposit_mode=mode,
                        relax_tol=1e-14 if precision == 0 else 1e-6)
    sid = sim.add_species(-1.0, 1.0, 1e-12, 1)
    sim.set_radiative_cooling(sid, K)
    u0 = math.sqrt(g0 * g0 - 1.0)
    sim.load_particles(sid, np.array([4.1]), np.array([4.2]), np.array([4.3]),
                       np.array([u0]), np.array([0.0]), np.array([0.0]))
    sim.load_fields(*_uniform_B(n, 1.0))
    sim.step(nsteps)
    assert sim.diagnostics()["status"] == 0
    p = sim.particles(sid)
    u = np.array([p["ux"][0], p["uy"][0], p["uz"][0]])
    ref = np.array([u0, 0.0, 0.0])
    for _ in range(nsteps):
        um = ref.copy()
        ref = orc.push(-dt, [0.0, 0.0, 0.0], [0.0, 0.0, 1.0], ref)
        ref = orc.radiate(K, dt, um, ref)
    assert np.abs(u - ref).max() <= tol * np.abs(ref).max(), (u, ref)
    gamma = math.sqrt(1.0 + u @ u)
    C = (g0 - 1.0) / (g0 + 1.0) * math.exp(-2.0 * K * nsteps * dt)
    exact = (1.0 + C) / (1.0 - C)
    assert abs(gamma - exact) <= 0.01 * (exact - 1.0), (gamma, exact)


def _plasma(orc, pp, precision, mode, K):
    L = pp_synth.random_particles((24, 16, 16), (0.5, 0.4, 0.45), 0.2, 3001, seed=5, u_scale=2.0)
    E, B = pp_synth.random_fields(L.n, 99, 0.05)
    B[2] = B[2] + 2.0
    gpu = H.gpu_sim(pp, L, precision, 3, deposit_mode=mode)
    for sid in range(len(L.species)):
        gpu.set_radiative_cooling(sid, K)
    gpu.load_fields(E, B)
    osim = orc.Simulation(L.n, L.d, L.dt, shape_order=3, relax_max_iter=2000)
    for s in L.species:
        osim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], rad=K)
    osim.load_fields(E, B)
    return L, gpu, osim


@pytest.mark.parametrize("precision,mode", [(0, 0), (1, 1), (1, 2)])
def test_cooling_plasma_parity(pp, orc, precision, mode):
    """Relativistic random particles (u ~ 2) in random fields plus B_z = 2 with
    K = 0.005: cooling changes the momenta by a few per cent per step.  Two
    steps, GPU against the oracle: FP64 at 1e-12; mixed at the tolerances of
    the uncooled mixed parity tests."""
    L, gpu, osim = _plasma(orc, pp, precision, mode, 0.005)
    gpu.step(2)
    osim.step(2)
    assert gpu.diagnostics()["status"] == 0
    if precision == 0:
        tol_f, tol_x, tol_u = 1e-12, 1e-12, 1e-12
    else:
        tol_f, tol_x, tol_u = 3e-5, 4e-6, 4e-6
    fe = H.field_errors(gpu, osim)
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(gpu.particles(s), osim.species[s], H.box(L))
        assert dpos <= tol_x and du <= tol_u, (s, dpos, du)
    for k, v in fe.items():
        assert v <= tol_f, (k, v, fe)


def test_cooling_survives_checkpoint(pp, orc, tmp_path):
    """The coefficient is part of the checkpoint: a restored run continues with
    cooling and matches the run that never stopped (FP64, particles matched by
    position since a restore re-sorts them); the same restore with cooling
    switched off does not."""
    L, a, _ = _plasma(orc, pp, 0, 0, 0.005)
    a.step(1)
    path = str(tmp_path / "cool.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    off = pp.Simulation.restore(path)
    for sid in range(len(L.species)):
        off.set_radiative_cooling(sid, 0.0)
    for sim in (a, b, off):
        sim.step(1)
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(b.particles(s), a.particles(s), H.box(L))
        assert dpos <= 1e-12 and du <= 1e-12, (s, dpos, du)
        _, du_off = H.particle_errors(off.particles(s), a.particles(s), H.box(L))
        assert du_off > 1e-4, (s, du_off)


def test_cooling_argument_checks(pp):
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2, shape_order=2, precision=1)
    sid = sim.add_species(-1.0, 1.0, 0.1, 10)
    for bad_sid, coef in ((sid + 1, 0.1), (-1, 0.1), (sid, -0.1), (sid, float("nan")), (sid, float("inf"))):
        with pytest.raises(RuntimeError):
            sim.set_radiative_cooling(bad_sid, coef)
    sim.set_radiative_cooling(sid, 0.0)
