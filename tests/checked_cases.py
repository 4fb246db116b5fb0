"""Cases run through the library twice by tests/test_gpu_checked.py: once with
the normal build and once, in a child process with PP_GB300_CHECKED=1, with the
bounds-checked build.  Prints one JSON line: per case the status of the last
diagnostics and the fields (E and B flattened)."""
import json
import sys

import numpy as np

import pp_synth


def _fields(sim):
    E, B, _ = sim.fields()
    return np.concatenate([a.ravel() for a in E + B]).tolist()


def run_cases():
    import paper_1211_4575_gb300 as pp
    from tests import gpu_helpers as H
    out = {}
    # mixed tiled, fast particles, no re-sort: many take the drift fallback
    L = pp_synth.random_particles((16, 16, 16), (0.5, 0.5, 0.5), 0.25, 4000, seed=77, u_scale=3.0)
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2, sort_interval=0)
    sim.load_fields(*pp_synth.random_fields(L.n, 3, 0.02))
    sim.step(12)
    out["tiled_drift"] = (sim.diagnostics()["status"], _fields(sim))
    # FP64 global kernels, every shape
    for shape in (1, 2, 3):
        L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=shape)
        sim = H.gpu_sim(pp, L, pp.PP_FP64, shape)
        sim.load_fields(*pp_synth.random_fields(L.n, 5, 0.05))
        sim.step(3)
        out[f"fp64_shape{shape}"] = (sim.diagnostics()["status"], _fields(sim))
    # direct current through the tiled kernel, and the 4th-order step
    L = pp_synth.thermal(n=(16, 16, 16), ppc=8, u_th=0.1, dx=0.1, dt=0.05, seed=5)
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2)
    sim.set_current_deposit(pp.PP_CURRENT_DIRECT)
    sim.step(4)
    out["tiled_direct"] = (sim.diagnostics()["status"], _fields(sim))
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2)
    sim.set_integrator(4)
    sim.step(3)
    out["tiled_step4"] = (sim.diagnostics()["status"], _fields(sim))
    # walls on x and y with an open end, an injector and a sliding window through
    # the tiled kernel: reflections, particles that leave, the unsorted tail,
    # window shifts
    L = pp_synth.random_particles((16, 16, 16), (0.5, 0.5, 0.5), 0.25, 4000, seed=78, u_scale=0.8)
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2, sort_interval=4, capacity_extra=6000,
                    boundary_x=pp.PP_BOUNDARY_WALLS, boundary_y=pp.PP_BOUNDARY_WALLS)
    sim.load_fields(*pp_synth.random_fields((32, 32, 16), 4, 0.02))
    sim.set_open_boundary(4, 0.2, 1.5)
    sim.set_injector(0, 1.0, (0.8, 0.0, 0.0), 0.1, 5)
    sim.set_sliding_window(0.5)
    sim.step(10)
    out["tiled_walls"] = (sim.diagnostics()["status"], _fields(sim))
    return out


if __name__ == "__main__":
    sys.path.insert(0, sys.argv[1])
    print(json.dumps(run_cases()))
