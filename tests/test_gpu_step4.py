"""GPU parity of the 4th-order symplectic step (Sec. III, the symmetric
fourth-order integrator: four kick-drift substeps) through pp_set_integrator,
against the FP64 oracle's four-substep step."""
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


def _pair(pp, orc, L, precision, shape, pusher=0, mode=0, rad=0.0, fields_seed=99):
    gpu = H.gpu_sim(pp, L, precision, shape, pusher=pusher, deposit_mode=mode)
    gpu.set_integrator(4)
    osim = orc.Simulation(L.n, L.d, L.dt, shape_order=shape, pusher=pusher, relax_tol=1e-14, relax_max_iter=2000,
                          integrator=4)
    for sid, s in enumerate(L.species):
        osim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], rad=rad)
        if rad:
            gpu.set_radiative_cooling(sid, rad)
    E, B = pp_synth.random_fields(L.n, fields_seed, 0.05)
    gpu.load_fields(E, B)
    osim.load_fields(E, B)
    return gpu, osim


def _compare(gpu, osim, L, tol_f, tol_x, tol_u):
    assert gpu.diagnostics()["status"] == 0
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(gpu.particles(s), osim.species[s], H.box(L))
        assert dpos <= tol_x and du <= tol_u, (s, dpos, du)
    fe = H.field_errors(gpu, osim)
    for k, v in fe.items():
        assert v <= tol_f, (k, v, fe)


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("pusher", [0, 1])
def test_step4_fp64_parity(pp, orc, shape, pusher):
    """Random particles (ragged 3001) in random fields on a non-cubic 20x12x9
    grid, two 4th-order steps (eight substeps, two with negative drifts): FP64
    to 1e-12 against the oracle."""
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=60 + shape + 3 * pusher)
    gpu, osim = _pair(pp, orc, L, 0, shape, pusher)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_step4_mixed_parity(pp, orc, mode):
    """Mixed form, global (1) and tiled (2) deposits on 24x16x16, two steps:
    fields 5e-5, positions and momenta 4e-6 (eight FP32 substeps)."""
    L = pp_synth.random_particles((24, 16, 16), (0.5, 0.4, 0.45), 0.2, 3001, seed=71)
    gpu, osim = _pair(pp, orc, L, 1, 3, mode=mode)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 5e-5, 4e-6, 4e-6)


def test_step4_with_radiative_cooling(pp, orc):
    """Cooling with the substeps' kick sizes (none in the drift-only first
    substep): relativistic particles, FP64 to 1e-12 against the oracle."""
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=5, u_scale=2.0)
    gpu, osim = _pair(pp, orc, L, 0, 3, rad=0.005)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


def _gyration_error(pp, h, order, u0=0.5):
    g0 = math.sqrt(1.0 + u0 * u0)
    om = 1.0 / g0
    n = int(round(4.0 * math.pi * g0 / h))
    T = n * h
    sim = pp.Simulation((8, 8, 8), (1.0, 1.0, 1.0), h, shape_order=3, alpha=0.5, precision=pp.PP_FP64,
                        relax_tol=1e-14)
    sim.set_integrator(order)
    sid = sim.add_species(-1.0, 1.0, 1e-10, 1)
    x0 = (3.3, 3.1, 4.2)
    t0 = 0.0 if order == 4 else -0.5 * h
    sim.load_particles(sid, np.array([x0[0]]), np.array([x0[1]]), np.array([x0[2]]),
                       np.array([u0 * math.cos(om * t0)]), np.array([u0 * math.sin(om * t0)]), np.array([0.0]))
    nx = 8
    E = [np.zeros((nx, nx, nx)) for _ in range(3)]
    B = [np.zeros((nx, nx, nx)) for _ in range(3)]
    B[2][...] = 1.0
    sim.load_fields(E, B)
    sim.step(n)
    p = sim.particles(sid)
    xe = x0[0] + u0 * math.sin(om * T)
    ye = x0[1] + u0 * (1.0 - math.cos(om * T))
    tu = T + t0
    dpos = max(abs((p["x"][0] - xe + 4.0) % 8.0 - 4.0), abs((p["y"][0] - ye + 4.0) % 8.0 - 4.0))
    du = max(abs(p["ux"][0] - u0 * math.cos(om * tu)), abs(p["uy"][0] - u0 * math.sin(om * tu)))
    return dpos, du


def test_step4_gyration_converges_at_fourth_order_on_gpu(pp):
    """The GPU's 4th-order step against the exact circle: halving dt divides the
    error by about 16 (the leap-frog's by about 4)."""
    e4 = [_gyration_error(pp, h, 4) for h in (0.4, 0.2)]
    e2 = [_gyration_error(pp, h, 2) for h in (0.4, 0.2)]
    for k in range(2):
        assert 13.0 < e4[0][k] / e4[1][k] < 17.0, e4
        assert 3.5 < e2[0][k] / e2[1][k] < 4.5, e2


def test_step4_order_survives_checkpoint(pp, orc, tmp_path):
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=81)
    a, _ = _pair(pp, orc, L, 0, 3)
    a.step(1)
    path = str(tmp_path / "s4.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    lf = pp.Simulation.restore(path)
    lf.set_integrator(2)
    for sim in (a, b, lf):
        sim.step(1)
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(b.particles(s), a.particles(s), H.box(L))
        assert dpos <= 1e-12 and du <= 1e-12, (s, dpos, du)
        _, du_lf = H.particle_errors(lf.particles(s), a.particles(s), H.box(L))
        assert du_lf > 1e-6, (s, du_lf)


def test_set_integrator_rejects_other_orders(pp):
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2, shape_order=2, precision=1)
    for order in (0, 1, 3, 6, -4):
        with pytest.raises(pp.PPError):
            sim.set_integrator(order)
    sim.set_integrator(4)
    sim.set_integrator(2)
