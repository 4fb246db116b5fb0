"""Shared helpers of the GPU parity tests: run the same seeded load through the
CUDA library (via the C ABI binding) and through the FP64 oracle, and compare
what is unique (fields element by element; particles as sets matched by
position, since the library keeps them in cell-sorted order)."""
import numpy as np


def gpu_sim(pp, L, precision, shape_order, field_order=6, alpha=0.55, pusher=0, relax_tol=None, sort_interval=20,
            deposit_mode=0, capacity_extra=0, relax_max_iter=400, stream=None, boundary_x=0, boundary_y=0,
            boundary_z=0):
    if relax_tol is None:
        relax_tol = 1e-14 if precision == pp.PP_FP64 else 1e-6
    sim = pp.Simulation(L.n, L.d, L.dt, field_order=field_order, alpha=alpha, shape_order=shape_order, pusher=pusher,
                        precision=precision, sort_interval=sort_interval, relax_max_iter=relax_max_iter,
                        relax_tol=relax_tol, deposit_mode=deposit_mode, stream=stream, boundary_x=boundary_x,
                        boundary_y=boundary_y, boundary_z=boundary_z)
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]) + capacity_extra)
        if len(s["x"]):
            sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    return sim


def oracle_sim(orc, L, shape_order, field_order=6, alpha=0.55, pusher=0, relax_tol=1e-14):
    sim = orc.Simulation(L.n, L.d, L.dt, field_order=field_order, alpha=alpha, shape_order=shape_order, pusher=pusher,
                         relax_tol=relax_tol, relax_max_iter=2000)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    return sim


def rel_err(a, b):
    """Norm-wise relative error max|a - b| / max|b| (absolute when b == 0)."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max() if b.size else 0.0
    d = np.abs(a - b).max() if b.size else 0.0
    return d / scale if scale > 0 else d


def field_errors(gpu, orc_sim):
    E, B, J = gpu.fields()
    out = {}
    for name, G, O in (("E", E, orc_sim.E), ("B", B, orc_sim.B), ("J", J, orc_sim.J)):
        num = max(np.abs(G[a] - O[a]).max() for a in range(3))
        den = max(np.abs(O[a]).max() for a in range(3))
        out[name] = num / den if den > 0 else num
    return out


def particle_errors(gpu_p, orc_p, box):
    """Match the two particle sets one to one by periodic nearest neighbour in
    position (the library keeps particles in cell-sorted order) and compare.
    Returns (max periodic position difference, relative momentum error)."""
    from scipy.spatial import cKDTree
    n = len(orc_p["x"])
    assert len(gpu_p["x"]) == n
    if n == 0:
        return 0.0, 0.0
    Lb = np.asarray(box, dtype=float)
    P = np.stack([np.mod(gpu_p[k], Lb[a]) for a, k in enumerate("xyz")], 1)
    O = np.stack([np.mod(orc_p[k], Lb[a]) for a, k in enumerate("xyz")], 1)
    P = np.minimum(P, np.nextafter(Lb, 0))
    O = np.minimum(O, np.nextafter(Lb, 0))
    _, j = cKDTree(O, boxsize=Lb).query(P, k=1)
    assert len(np.unique(j)) == n, "particle sets do not match one to one"
    d = P - O[j]
    d = (d + 0.5 * Lb) % Lb - 0.5 * Lb
    dpos = np.abs(d).max()
    du = max(np.abs(gpu_p[k] - orc_p[k][j]).max() for k in ("ux", "uy", "uz"))
    us = max(np.abs(orc_p[k]).max() for k in ("ux", "uy", "uz"))
    return dpos, (du / us if us > 0 else du)


def box(L):
    return tuple(L.n[a] * L.d[a] for a in range(3))
