"""z-slab decomposition of one run (paper_1211_4575_gb300.parallel, Sec. IX)
on CPU ranks over gloo, with the FP64 oracle as each rank's compute: after
several steps in which particles cross the slab boundaries (and the periodic
box edge), the fields of every rank and the union of the ranks' particles
equal those of the same run on one domain to 1e-12 (the ranks' currents are
summed in another order; nothing else differs)."""
import os
import socket

import numpy as np
import pytest

import pp_synth

STEPS = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _load():
    # fast particles: many cross a slab boundary (and z = 0) within the steps
    L = pp_synth.random_particles((8, 8, 16), (0.5, 0.5, 0.5), 0.2, 1500, seed=77, u_scale=0.8)
    extra = pp_synth.random_particles((8, 8, 16), (0.5, 0.5, 0.5), 0.2, 900, seed=78, u_scale=0.5, q=1.0, m=4.0)
    L.species.append(extra.species[0])
    return L


KW = dict(field_order=6, alpha=0.55, shape_order=3, relax_tol=1e-14, relax_max_iter=2000)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1211_4575_gb300 import parallel
    from tests.slab_oracle import OracleSlab
    oracle.build()
    L = _load()
    sim = OracleSlab(oracle, L.n, L.d, L.dt, **KW)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"])
    bounds = parallel.slab_bounds(L.n[2], L.d[2], world)
    sl = parallel.Slab(sim, rank, bounds, len(L.species))
    parallel.load([sl], L.species)
    comm = parallel.TorchComm()
    moved = 0
    for _ in range(STEPS):
        before = [sim.count(s) for s in range(len(L.species))]
        parallel.step([sl], comm)
        moved += sum(abs(sim.count(s) - b) for s, b in enumerate(before))
    kin, count = parallel.kinetic_and_count([sl], comm)
    parts = [{k: sim.o.species[s][k] for k in ("x", "y", "z", "ux", "uy", "uz")} for s in range(len(L.species))]
    inside = all(((p["z"] >= bounds[rank][0]) & (p["z"] < bounds[rank][1])).all() for p in parts)
    gathered = [None] * world
    dist.gather_object((rank, [a.copy() for a in sim.o.E], [a.copy() for a in sim.o.B], [a.copy() for a in sim.o.J],
                        parts, moved, inside, count), gathered if rank == 0 else None, dst=0)
    if rank == 0:
        out.put(gathered)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slab_decomposition_equals_single_domain_over_gloo(orc, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the same run on one domain
    L = _load()
    ref = orc.Simulation(L.n, L.d, L.dt, **KW)
    for s in L.species:
        ref.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    for _ in range(STEPS):
        ref.deposit()
        ref.field_update()
    assert sum(g[5] for g in gathered) > 20, "too few particles changed slab to test migration"
    assert all(g[6] for g in gathered), "a rank holds a particle outside its slab"
    assert gathered[0][7] == L.n_particles
    for rank, E, B, J, parts, _, _, _ in gathered:
        for name, G, O in (("E", E, ref.E), ("B", B, ref.B), ("J", J, ref.J)):
            err = max(np.abs(G[a] - O[a]).max() for a in range(3)) / max(np.abs(O[a]).max() for a in range(3))
            assert err <= 1e-12, (world, rank, name, err)
    from scipy.spatial import cKDTree
    box = np.array([L.n[a] * L.d[a] for a in range(3)])
    for s in range(len(L.species)):
        P = {k: np.concatenate([g[4][s][k] for g in gathered]) for k in ("x", "y", "z", "ux", "uy", "uz")}
        O = ref.species[s]
        assert len(P["x"]) == len(O["x"])
        A = np.stack([P["x"], P["y"], P["z"]], 1) % box
        Bq = np.stack([O["x"], O["y"], O["z"]], 1) % box
        _, j = cKDTree(Bq, boxsize=box).query(A, k=1)
        assert len(np.unique(j)) == len(j)
        d = (A - Bq[j] + 0.5 * box) % box - 0.5 * box
        assert np.abs(d).max() <= 1e-12 * box.max()
        us = max(np.abs(O[k]).max() for k in ("ux", "uy", "uz"))
        assert max(np.abs(P[k] - O[k][j]).max() for k in ("ux", "uy", "uz")) <= 1e-12 * us


def test_slab_bounds_and_owner():
    from paper_1211_4575_gb300 import parallel
    b = parallel.slab_bounds(10, 0.5, 3)
    assert b == [(0.0, 2.0), (2.0, 3.5), (3.5, 5.0)]
    assert list(parallel.owner([0.0, 1.99, 2.0, 3.49, 3.5, 4.99], b)) == [0, 0, 1, 1, 2, 2]
    with pytest.raises(ValueError):
        parallel.slab_bounds(4, 1.0, 5)
