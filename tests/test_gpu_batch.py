"""Batched / served form: independent runs admitted into slots by device-memory
budget and advanced together give the same result as each run alone."""
import numpy as np
import pytest

from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as m
    return m


def _requests():
    return [dict(arrival=0.0, kind="two-stream", n=16, ppc=8, beta=0.2, u_th=0.05, plasma="pair", shape=3, steps=9,
                 seed=11),
            dict(arrival=0.0, kind="weibel", n=8, ppc=12, beta=0.5, u_th=0.1, plasma="ion", shape=2, steps=5, seed=12),
            dict(arrival=0.0, kind="two-stream", n=24, ppc=4, beta=0.3, u_th=0.02, plasma="pair", shape=3, steps=7,
                 seed=13)]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 5e-5)])
def test_each_result_same_alone_and_in_the_mix(pp, precision, tol):
    from paper_1211_4575_gb300 import serving
    reqs = _requests()
    alone, ra = serving.sequential(reqs, precision=precision, keep=True)
    mixed, rm = serving.serve(reqs, budget_bytes=8 << 30, max_slots=4, chunk=2, precision=precision, keep=True)
    assert alone["requests"] == mixed["requests"] == 3
    by_seed = {r["seed"]: s for r, s in ra}
    for req, sim in rm:
        ref = by_seed[req["seed"]]
        E1, B1, _ = sim.fields()
        E0, B0, _ = ref.fields()
        assert max(H.rel_err(E1[a], E0[a]) for a in range(3)) <= tol
        assert max(H.rel_err(B1[a], B0[a]) for a in range(3)) <= tol
        for s in range(2):
            p1, p0 = sim.particles(s), ref.particles(s)
            dpos, du = H.particle_errors(p1, p0, tuple(req["n"] * 0.5 for _ in range(3)))
            assert dpos <= tol and du <= tol
        d1, d0 = sim.diagnostics(), ref.diagnostics()
        assert d1["step"] == d0["step"] == req["steps"]
        sim.close()
        ref.close()


def test_fused_rounds_same_as_alone(pp):
    """Fused rounds (one persistent particle launch over the tiles of every
    running slot, PCS and TSC runs in two groups): each result equals the run
    alone to the mixed form's round-off (the flush of a tile's current into
    the mesh is an FP32 atomic sum, order-dependent)."""
    from paper_1211_4575_gb300 import serving
    reqs = [dict(r, n=((r["n"] + 7) // 8) * 8) for r in _requests()]   # meshes of multiples of 8
    alone, ra = serving.sequential(reqs, precision=pp.PP_MIXED32, keep=True)
    mixed, rm = serving.serve(reqs, budget_bytes=8 << 30, max_slots=4, chunk=2, precision=pp.PP_MIXED32, keep=True,
                              fused=True)
    assert mixed["requests"] == 3
    by_seed = {r["seed"]: s for r, s in ra}
    for req, sim in rm:
        ref = by_seed[req["seed"]]
        E1, B1, _ = sim.fields()
        E0, B0, _ = ref.fields()
        assert max(H.rel_err(E1[a], E0[a]) for a in range(3)) <= 5e-5
        assert max(H.rel_err(B1[a], B0[a]) for a in range(3)) <= 5e-5
        for s in range(2):
            dpos, du = H.particle_errors(sim.particles(s), ref.particles(s), tuple(req["n"] * 0.5 for _ in range(3)))
            assert dpos <= 5e-5 and du <= 5e-5
        assert sim.diagnostics()["step"] == ref.diagnostics()["step"] == req["steps"]
        sim.close()
        ref.close()


def test_admission_by_budget_and_slots(pp):
    import pp_synth
    L = pp_synth.run_load(_requests()[0])

    def make():
        sim = pp.Simulation(L.n, L.d, L.dt, shape_order=3, precision=pp.PP_MIXED32)
        for s in L.species:
            sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]))
            sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
        return sim

    a, b, c = make(), make(), make()
    need = a.device_bytes()
    assert need > 0
    # the estimate a server takes before building equals what the built run holds
    assert pp.estimate_device_bytes(L.n, [len(s["x"]) for s in L.species], pp.PP_MIXED32) == need
    assert pp.estimate_device_bytes(L.n, pp_synth.run_counts(_requests()[0]), pp.PP_MIXED32) == need
    batch = pp.Batch(int(2.5 * need), max_slots=8)
    sa = batch.admit(a, 3)
    sb = batch.admit(b, 1)
    assert sa is not None and sb is not None
    assert batch.admit(c, 2) is None                 # over the device-memory budget
    assert batch.used() == (2 * need, 2)
    import time
    states = {}
    t_end = time.time() + 30.0
    while len(states) < 2 and time.time() < t_end:   # polling never blocks: wait for the device
        batch.advance(1)
        for s in (sa, sb):
            if s in states:
                continue
            st, done = batch.poll(s)
            if st != pp.PP_BATCH_RUNNING:
                states[s] = (st, done)
        time.sleep(0.01)
    assert states[sa] == (pp.PP_BATCH_DONE, 3) and states[sb] == (pp.PP_BATCH_DONE, 1)
    assert batch.used() == (0, 0)
    assert batch.admit(c, 2) is not None             # capacity came back
    batch.close()


def test_autotuner_picks_a_candidate_and_keeps_physics(pp):
    import pp_synth
    from paper_1211_4575_gb300 import autotune
    L = pp_synth.thermal(n=(16, 16, 16), ppc=8, dx=0.1, dt=0.05, seed=3)
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
    best, timings = autotune.autotune(sim, sort_intervals=(2, 4), steps=4, use_cache=False)
    # the per-step sorted mode once, the tiled and global modes at each interval
    assert best in timings and len(timings) == 5 and (1, pp.PP_DEPOSIT_CELLS) in timings
    g, _ = sim.grid()
    assert (g.sort_interval, g.deposit_mode) == best
    d = sim.diagnostics()
    assert d["status"] == 0 and d["step"] == 20
    assert d["gauss_drift_max"] <= 2e-5 * d["rho_max"]
    with pytest.raises(pp.PPError):
        H.gpu_sim(pp, pp_synth.thermal(n=(12, 12, 12), ppc=2, dx=0.1, dt=0.05), pp.PP_MIXED32, 3).set_tuning(
            20, pp.PP_DEPOSIT_TILED)
