"""Step graphs (pp_set_graphs): a step captured as a CUDA graph and replayed
gives the eager step's results, through sorts, the J / J' alternation, the
4th-order substeps and parameter changes that drop the captures."""
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


def _sim(pp, L, precision, shape, graphs, sort_interval, extra=0, **kw):
    import torch
    stream = torch.cuda.Stream()
    sim = pp.Simulation(L.n, L.d, L.dt, shape_order=shape, precision=precision, sort_interval=sort_interval,
                        relax_tol=1e-14 if precision == pp.PP_FP64 else 1e-6, stream=stream.cuda_stream, **kw)
    sim._keep_stream = stream
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]) + extra)
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    if graphs:
        sim.set_graphs(True)
    return sim


def _compare(a, b, L, tol_f, tol_x, tol_u):
    Ea, Ba, Ja = a.fields()
    Eb, Bb, Jb = b.fields()
    for X, Y in ((Ea, Eb), (Ba, Bb), (Ja, Jb)):
        assert max(H.rel_err(X[k], Y[k]) for k in range(3)) <= tol_f
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(a.particles(s), b.particles(s), H.box(L))
        assert dpos <= tol_x and du <= tol_u, (s, dpos, du)


def test_graphs_fp64_match_eager_through_sorts(pp):
    """C1-like two-stream, FP64, a sort every 3 steps: 20 graph steps equal 20
    eager steps to 1e-12, and most steps are replays of earlier captures."""
    L = pp_synth.two_stream()
    eager = _sim(pp, L, pp.PP_FP64, 2, False, 3)
    graph = _sim(pp, L, pp.PP_FP64, 2, True, 3)
    for _ in range(20):
        eager.step(1)
        graph.step(1)
    _compare(graph, eager, L, 1e-12, 1e-12, 1e-12)
    cap, rep = graph.graph_stats()
    assert cap + rep == 20 and cap <= 8 and rep >= 12, (cap, rep)
    assert eager.graph_stats() == (0, 0)
    assert graph.diagnostics()["step"] == 20


def test_graphs_mixed_tiled_thermal(pp):
    """Mixed form, tiled kernel, thermal PCS on 24^3 with a sort every 4 steps,
    30 steps.  Both runs flush their current windows with FP32 atomics in
    arbitrary order, so they agree to FP32 round-off grown over the run."""
    L = pp_synth.thermal(n=(24, 24, 24), ppc=8, u_th=0.1, dx=0.1, dt=0.05, seed=1212)
    eager = _sim(pp, L, pp.PP_MIXED32, 3, False, 4)
    graph = _sim(pp, L, pp.PP_MIXED32, 3, True, 4)
    eager.step(30)
    graph.step(30)
    assert graph.diagnostics()["status"] == 0
    _compare(graph, eager, L, 1e-4, 1e-5, 1e-4)
    cap, rep = graph.graph_stats()
    assert rep >= 22, (cap, rep)


def test_graphs_fourth_order_with_cooling(pp):
    """The four substeps and cooling inside one capture: FP64, 6 steps with a
    sort every 2, against eager to 1e-12."""
    L = pp_synth.random_particles((16, 8, 8), (0.5, 0.4, 0.45), 0.2, 2001, seed=9, u_scale=1.0)
    sims = []
    for graphs in (False, True):
        s = _sim(pp, L, pp.PP_FP64, 3, graphs, 2)
        s.set_integrator(4)
        s.set_radiative_cooling(0, 0.005)
        E, B = pp_synth.random_fields(L.n, 4, 0.05)
        s.load_fields(E, B)
        s.step(6)
        sims.append(s)
    _compare(sims[1], sims[0], L, 1e-12, 1e-12, 1e-12)
    assert sims[1].graph_stats()[1] >= 2


def test_parameter_changes_drop_captures(pp):
    """Changing the integrator, the cooling and the particle load between steps
    re-captures, and the result still equals the eager sequence."""
    L = pp_synth.random_particles((16, 8, 8), (0.5, 0.4, 0.45), 0.2, 1500, seed=12)
    extra = pp_synth.random_particles((16, 8, 8), (0.5, 0.4, 0.45), 0.2, 300, seed=13)
    caps = []
    sims = []
    for graphs in (False, True):
        s = _sim(pp, L, pp.PP_FP64, 2, graphs, 3, extra=300)
        s.step(4)
        c0 = s.graph_stats()[0]
        s.set_integrator(4)
        s.step(2)
        c1 = s.graph_stats()[0]
        s.set_radiative_cooling(0, 0.01)
        s.step(2)
        c2 = s.graph_stats()[0]
        sp = extra.species[0]
        s.load_particles(0, sp["x"], sp["y"], sp["z"], sp["ux"], sp["uy"], sp["uz"])
        s.step(3)
        c3 = s.graph_stats()[0]
        caps.append((c0, c1, c2, c3))
        sims.append(s)
    _compare(sims[1], sims[0], L, 1e-12, 1e-12, 1e-12)
    c0, c1, c2, c3 = caps[1]
    assert c0 < c1 < c2 < c3, caps


def test_graphs_need_a_stream_and_skip_profiling(pp):
    L = pp_synth.random_particles((8, 8, 8), (0.5, 0.5, 0.5), 0.2, 200, seed=3)
    legacy = pp.Simulation(L.n, L.d, L.dt, shape_order=2, precision=pp.PP_MIXED32, stream=None)
    if not legacy.grid()[0].stream:   # torch's current stream is the legacy default here
        with pytest.raises(pp.PPError):
            legacy.set_graphs(True)
    sim = _sim(pp, L, pp.PP_MIXED32, 2, True, 0)
    # per-step sorted kernel: the first step starts from the load's sort; after
    # it every step sorts from the keys of the last pass, and J / J' and the two
    # particle buffers alternate: three captures, then a replay
    sim.step(4)
    assert sim.graph_stats() == (3, 1)
    sim.profile_enable(True)
    sim.step(3)
    sim.profile_enable(False)
    assert sim.graph_stats() == (3, 1)    # profiled steps run eagerly
    sim.step(1)
    assert sim.graph_stats() == (3, 2)
