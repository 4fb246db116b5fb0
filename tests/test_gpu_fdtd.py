"""GPU parity of the explicit FDTD field solver (the cold-beam comparison of
Sec. VIII) through pp_set_field_solver, against the FP64 oracle's leap-frog
and the scheme's closed-form dispersion."""
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


def _pair(pp, orc, L, precision, shape, forder=6, mode=0, integrator=2):
    gpu = H.gpu_sim(pp, L, precision, shape, field_order=forder, deposit_mode=mode)
    gpu.set_field_solver(pp.PP_FIELD_EXPLICIT)
    gpu.set_integrator(integrator)
    osim = orc.Simulation(L.n, L.d, L.dt, field_order=forder, shape_order=shape, field_solver=orc.EXPLICIT,
                          integrator=integrator)
    for s in L.species:
        osim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    E, B = pp_synth.random_fields(L.n, 17, 0.05)
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
@pytest.mark.parametrize("forder", [2, 4, 6])
def test_explicit_fp64_parity(pp, orc, shape, forder):
    """Random particles (ragged 3001) in random fields on 20x12x9 (dt 0.1 under
    the leap-frog limit), three steps: FP64 to 1e-12 against the oracle."""
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.1, 3001, seed=90 + 3 * shape + forder)
    gpu, osim = _pair(pp, orc, L, 0, shape, forder)
    gpu.step(3)
    osim.step(3)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_explicit_mixed_parity(pp, orc, mode):
    """Mixed form, global (1) and tiled (2) deposits on 24x16x16, three steps:
    fields 3e-5, positions and momenta 2e-6 (no relaxation tolerance here)."""
    L = pp_synth.random_particles((24, 16, 16), (0.5, 0.4, 0.45), 0.1, 3001, seed=95)
    gpu, osim = _pair(pp, orc, L, 1, 3, mode=mode)
    gpu.step(3)
    osim.step(3)
    _compare(gpu, osim, L, 3e-5, 2e-6, 2e-6)


def test_explicit_with_fourth_order_step(pp, orc):
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.1, 2001, seed=97)
    gpu, osim = _pair(pp, orc, L, 0, 3, integrator=4)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


def test_explicit_vacuum_dispersion_on_gpu(pp, orc):
    """FP64 on the GPU: a standing vacuum mode follows e(n+1) + e(n-1) =
    2 cos(phi) e(n), cos(phi) = 1 - (dt K(k))^2 / 2, with no damping."""
    nx, dx, dt, mode = 16, 0.5, 0.2, 3
    sim = pp.Simulation((nx, 2, 2), (dx, dx, dx), dt, field_order=6, precision=pp.PP_FP64)
    sim.set_field_solver(pp.PP_FIELD_EXPLICIT)
    k = 2 * np.pi * mode / (nx * dx)
    x = np.arange(nx) * dx
    E = [np.zeros((2, 2, nx)) for _ in range(3)]
    B = [np.zeros((2, 2, nx)) for _ in range(3)]
    E[1][...] = np.cos(k * x)
    sim.load_fields(E, B)
    basis = np.broadcast_to(np.cos(k * x), (2, 2, nx))
    e = []
    for _ in range(40):
        Eg, _, _ = sim.fields()
        e.append((Eg[1] * basis).sum() / (basis * basis).sum())
        sim.step(1)
    e = np.array(e)
    kc = orc.fd_coeffs(6)
    K = (2 / dx) * (kc[0] * np.sin(k * dx / 2) + kc[1] * np.sin(3 * k * dx / 2) + kc[2] * np.sin(5 * k * dx / 2))
    cphi = 1.0 - (dt * K) ** 2 / 2.0
    assert np.abs(e[2:] + e[:-2] - 2 * cphi * e[1:-1]).max() < 1e-12
    assert np.abs(e).max() > 0.5


def test_explicit_limit_and_checkpoint(pp, orc, tmp_path):
    # dt above the leap-frog limit (0.5 * dx here) is refused
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.25, precision=pp.PP_FP64)
    with pytest.raises(pp.PPError):
        sim.set_field_solver(pp.PP_FIELD_EXPLICIT)
    with pytest.raises(pp.PPError):
        sim.set_field_solver(7)
    # the solver is part of the checkpoint
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.1, 1000, seed=98)
    a, _ = _pair(pp, orc, L, 0, 2)
    a.step(1)
    path = str(tmp_path / "fdtd.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    imp = pp.Simulation.restore(path)
    imp.set_field_solver(pp.PP_FIELD_IMPLICIT)
    for s in (a, b, imp):
        s.step(2)
    Ea, _, _ = a.fields()
    Eb, _, _ = b.fields()
    Ei, _, _ = imp.fields()
    assert max(H.rel_err(Eb[k], Ea[k]) for k in range(3)) <= 1e-12
    assert max(H.rel_err(Ei[k], Ea[k]) for k in range(3)) > 1e-6
