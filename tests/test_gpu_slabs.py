"""z-slab decomposition on the GPU (paper_1211_4575_gb300.parallel): one
library context per slab, all in this process on one GPU, their currents
summed on the device (LocalComm: the same driver a multi-GPU run uses with
NCCL) and their leaving particles moved through pp_extract_particles and
pp_load_particles.  After several steps with migration the fields of every
slab and the union of the slabs' particles equal the single-domain run of the
library (FP64: 1e-12; mixed form: its FP32 tolerances) and the FP64 oracle."""
import numpy as np
import pytest

import pp_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
STEPS = 6


@pytest.fixture(scope="module")
def pp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4575_gb300 as m
    from paper_1211_4575_gb300 import build
    build.build()
    return m


def _load():
    L = pp_synth.random_particles((8, 8, 16), (0.5, 0.5, 0.5), 0.2, 1500, seed=77, u_scale=0.8)
    extra = pp_synth.random_particles((8, 8, 16), (0.5, 0.5, 0.5), 0.2, 900, seed=78, u_scale=0.5, q=1.0, m=4.0)
    L.species.append(extra.species[0])
    return L


def _slab_run(pp, L, precision, world):
    import torch
    from paper_1211_4575_gb300 import parallel
    bounds = parallel.slab_bounds(L.n[2], L.d[2], world)
    slabs = []
    for r in range(world):
        sim = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3, precision=precision,
                            relax_tol=1e-14 if precision == pp.PP_FP64 else 1e-6, relax_max_iter=2000)
        for s in L.species:
            sim.add_species(s["q"], s["m"], s["w"], L.n_particles)
        slabs.append(parallel.Slab(sim, r, bounds, len(L.species)))
    parallel.load(slabs, L.species)
    comm = parallel.LocalComm(world)
    dev = torch.device("cuda", torch.cuda.current_device())
    moved = 0
    for _ in range(STEPS):
        before = [[sl.sim.count(s) for s in range(len(L.species))] for sl in slabs]
        parallel.step(slabs, comm, device=dev)
        moved += sum(abs(sl.sim.count(s) - b[s]) for sl, b in zip(slabs, before) for s in range(len(L.species)))
    return slabs, bounds, moved


def _union(slabs, s):
    ps = [sl.sim.particles(s) for sl in slabs]
    return {k: np.concatenate([p[k] for p in ps]) for k in ("x", "y", "z", "ux", "uy", "uz")}


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_slabs_equal_single_domain(pp, orc, world, precision):
    from paper_1211_4575_gb300 import parallel
    L = _load()
    slabs, bounds, moved = _slab_run(pp, L, precision, world)
    assert moved > 20
    one = H.gpu_sim(pp, L, precision, 3)
    osim = H.oracle_sim(orc, L, 3)
    for _ in range(STEPS):
        one.deposit()
        one.field_update()
        osim.step(1)
    tol = (1e-12, 1e-12, 1e-12) if precision == pp.PP_FP64 else (3e-5 * STEPS, 2e-6 * STEPS, 2e-6 * STEPS)
    for sl in slabs:
        assert sl.sim.diagnostics()["status"] == 0
        for ref in (one, osim):
            fe = H.field_errors(sl.sim, ref) if ref is osim else _field_errors(sl.sim, one)
            for k, v in fe.items():
                assert v <= tol[0], (world, precision, sl.rank, k, v)
        for s in range(len(L.species)):
            p = sl.sim.particles(s)
            lo, hi = bounds[sl.rank]
            assert ((p["z"] >= lo) & (p["z"] < hi)).all()
    for s in range(len(L.species)):
        U = _union(slabs, s)
        for ref_p in (one.particles(s), osim.species[s]):
            dpos, du = H.particle_errors(U, ref_p, H.box(L))
            assert dpos <= tol[1] and du <= tol[2], (world, precision, s, dpos, du)
    kin, count = parallel.kinetic_and_count(slabs, parallel.LocalComm(world))
    assert count == L.n_particles
    d1 = one.diagnostics()
    assert np.allclose(kin, d1["kinetic"], rtol=1e-10 if precision == pp.PP_FP64 else 1e-5)


def _field_errors(a, b):
    Ea, Ba, Ja = a.fields()
    Eb, Bb, Jb = b.fields()
    out = {}
    for name, G, O in (("E", Ea, Eb), ("B", Ba, Bb), ("J", Ja, Jb)):
        out[name] = max(np.abs(G[k] - O[k]).max() for k in range(3)) / max(np.abs(O[k]).max() for k in range(3))
    return out


def test_extract_arguments(pp):
    L = _load()
    sim = H.gpu_sim(pp, L, pp.PP_FP64, 3)
    with pytest.raises(pp.PPError):
        sim.extract_particles(0)            # no slab declared
    with pytest.raises(pp.PPError):
        sim.set_slab(2.0, 1.0)
    sim.set_slab(1.0, 3.0)
    n0 = sim.count(0)
    left = sim.extract_particles(0)
    assert sim.count(0) + len(left["x"]) == n0
    assert ((left["z"] < 1.0) | (left["z"] >= 3.0)).all()
    p = sim.particles(0)
    assert ((p["z"] >= 1.0) & (p["z"] < 3.0)).all()
