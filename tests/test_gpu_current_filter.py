"""GPU parity of the direct current eq:jj2 (pp_set_current_deposit) and the
divergence filter (pp_set_divergence_filter), the cold-beam study's other
variants, against the FP64 oracle."""
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


def _pair(pp, orc, L, precision, shape, pusher=0, mode=0, current=1, passes=0, interval=1, fields=True,
          sort_interval=20, stream=None):
    gpu = H.gpu_sim(pp, L, precision, shape, pusher=pusher, deposit_mode=mode, sort_interval=sort_interval,
                    stream=stream)
    gpu.set_current_deposit(current)
    gpu.set_divergence_filter(passes, interval)
    osim = orc.Simulation(L.n, L.d, L.dt, shape_order=shape, pusher=pusher, relax_tol=1e-14, relax_max_iter=2000,
                          current_mode=current, filter_passes=passes, filter_interval=interval)
    for s in L.species:
        osim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    if fields:
        E, B = pp_synth.random_fields(L.n, 23, 0.05)
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
def test_direct_current_fp64_parity(pp, orc, shape, pusher):
    """eq:jj2 through the FP64 kernels: random particles (ragged 3001) in random
    fields on 20x12x9, two steps, 1e-12 against the oracle."""
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=120 + shape + 3 * pusher)
    gpu, osim = _pair(pp, orc, L, 0, shape, pusher)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_direct_current_mixed_parity(pp, orc, mode):
    """Mixed form, global (1) and tiled (2): fields 3e-5, positions and momenta 2e-6."""
    L = pp_synth.random_particles((24, 16, 16), (0.5, 0.4, 0.45), 0.2, 3001, seed=131)
    gpu, osim = _pair(pp, orc, L, 1, 3, mode=mode)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 3e-5, 2e-6, 2e-6)


@pytest.mark.parametrize("current,passes,interval", [(1, 5, 1), (0, 1, 2)])
def test_filter_fp64_parity(pp, orc, current, passes, interval):
    """The direct current with 5 filter passes every step (the original method),
    and the charge-conserving current with one pass every second step (the
    periodic filter): C1 two-stream, FP64, 4 steps, 1e-12."""
    L = pp_synth.two_stream()
    gpu, osim = _pair(pp, orc, L, 0, 2, current=current, passes=passes, interval=interval, fields=False)
    gpu.step(4)
    osim.step(4)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


def test_filter_mixed_tiled_parity(pp, orc):
    L = pp_synth.thermal(n=(24, 24, 24), ppc=4, u_th=0.1, dx=0.1, dt=0.05, seed=1212)
    gpu, osim = _pair(pp, orc, L, 1, 3, mode=2, current=1, passes=3, interval=1, fields=False)
    gpu.step(3)
    osim.step(3)
    _compare(gpu, osim, L, 5e-5, 2e-6, 2e-6)


def test_filter_holds_gauss_law_for_the_direct_current(pp):
    """Mixed form, thermal plasma with the direct current: without the filter
    the Gauss residual drifts; 10 passes per step keep it far smaller."""
    L = pp_synth.thermal(n=(24, 24, 24), ppc=8, u_th=0.1, dx=0.1, dt=0.05, seed=1212)
    drift = {}
    for passes in (0, 10):
        sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
        sim.set_current_deposit(pp.PP_CURRENT_DIRECT)
        sim.set_divergence_filter(passes, 1)
        sim.step(10)
        d = sim.diagnostics()
        assert d["status"] == 0
        drift[passes] = d["gauss_max"] / d["rho_max"]
    assert drift[10] < 0.1 * drift[0], drift


def test_graphs_through_filtered_steps(pp, orc):
    import torch
    L = pp_synth.two_stream()
    sims = []
    for graphs in (False, True):
        s = torch.cuda.Stream()
        gpu, _ = _pair(pp, orc, L, 0, 2, current=1, passes=2, interval=3, fields=False, sort_interval=4,
                       stream=s.cuda_stream)
        gpu._keep = s
        if graphs:
            gpu.set_graphs(True)
        gpu.step(13)
        sims.append(gpu)
    E0, B0, _ = sims[0].fields()
    E1, B1, _ = sims[1].fields()
    assert max(H.rel_err(E1[a], E0[a]) for a in range(3)) <= 1e-12
    assert max(H.rel_err(B1[a], B0[a]) for a in range(3)) <= 1e-12
    assert sims[1].graph_stats()[1] > 0


def test_current_and_filter_arguments_and_checkpoint(pp, orc, tmp_path):
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2, precision=pp.PP_FP64)
    for bad in (-1, 2):
        with pytest.raises(pp.PPError):
            sim.set_current_deposit(bad)
    for passes, interval in ((-1, 1), (1, 0)):
        with pytest.raises(pp.PPError):
            sim.set_divergence_filter(passes, interval)
    L = pp_synth.two_stream(n=(8, 8, 8))
    a, _ = _pair(pp, orc, L, 0, 2, current=1, passes=3, interval=1, fields=False)
    a.step(1)
    path = str(tmp_path / "cf.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    plain = pp.Simulation.restore(path)
    plain.set_current_deposit(pp.PP_CURRENT_CONSERVING)
    plain.set_divergence_filter(0, 1)
    for s in (a, b, plain):
        s.step(2)
    Ea, _, _ = a.fields()
    Eb, _, _ = b.fields()
    Ep, _, _ = plain.fields()
    assert max(H.rel_err(Eb[k], Ea[k]) for k in range(3)) <= 1e-12
    assert max(H.rel_err(Ep[k], Ea[k]) for k in range(3)) > 1e-6
