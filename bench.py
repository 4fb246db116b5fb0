#!/usr/bin/env python
"""Throughput benchmark of the GB300 Photon-Plasma particle step.

One "step" is one full leap-frog step of the library (pp_step): the cell sort
(every step for the per-step sorted kernel), the fused gather -> push -> move
-> charge-conserving deposit kernel over every species, ghost fold, 6th-order
current solve and the implicit field update.  Default workload: the
mixed-precision beam configuration, a cold Gamma = 10 beam streaming through a
thermal electron-ion background (m_i/m_e = 25, u_th = 0.01c) on 256 x 128 x 128
cells, 16 macro-particles per cell per species per population (268,435,456
particles), PCS shapes, 6th-order fields, int32 cell + FP32 offset.
`--workload thermal` runs the 128^3 numerical-heating pair plasma (32 per cell
per species, 134,217,728 particles).  Inputs are seeded synthetic loads
(pp_synth).

Prints one JSON line (rank 0).  Multi-GPU: every rank advances its own
independent plasma (replicas, weak scaling); no collective on the data path.
The cpu_baseline leg times the FP64 oracle on a 32^3 crop of the workload
(the same per-cell load on a periodic 32^3 box) and states the GPU's error
against it on that crop.  `--impl reference` times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit)"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = 56   # mixed form: (int32 cell + 3 fp32 offsets + 3 fp32 momenta) read + written

# ncu figures of the per-step sorted particle kernel, per particle, from one
# capture of one launch on a small case of each workload with the workload's
# per-cell load (beam: 128x64x64 cells; thermal: 64^3 cells): DRAM traffic
# (dram__bytes_read.sum + dram__bytes_write.sum; traffic grows with the
# particle count), warp-instructions (smsp__inst_executed.sum) and the
# limiter the capture shows.  An entry holds only while the kernel's sources
# are the ones it was taken on (sha256 below); otherwise the line reports
# traffic, limiter and issue as null.
PROFILED = {
    "beam": {"bytes_per_particle": 64.55, "warp_inst_per_particle": 100.2,
             "limiter": "instruction issue (63.0 % of issue slots busy; LSU 41.0 %, FMA 37.0 % of peak; "
                        "DRAM 6.1 %)"},
    "thermal": {"bytes_per_particle": 66.23, "warp_inst_per_particle": 94.6,
                "limiter": "instruction issue (57.3 % of issue slots busy; LSU 39.4 %, FMA 32.2 % of peak; "
                           "DRAM 5.3 %)"},
}
PROFILED_SOURCES = {
    "paper_1211_4575_gb300/csrc/pp_cells.cu": "16c7f12cf0f9e413eae8c402bdf089400dd7af4e2ce7593d6ed90713baf03ed6",
    "paper_1211_4575_gb300/csrc/pp_internal.cuh": "00cb3fc2fa3f0515a11f11b42e8eb92fa4d4d124135cefaf834886bc46b91cb9",
    "paper_1211_4575_gb300/csrc/pp_particle_common.cuh": "6805ab903ef2be60e620b6059392d7afd2da3fd0f9a098f8dbf04858b8b05717",
    "paper_1211_4575_gb300/csrc/pp_tma.cuh": "e0ac1f2401ee66da9f6509e7830a148f7aadb33c4eab9f1a62bf6f1a7995817c",
}


def _digest(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profiled(a):
    """The ncu figures of this workload's capture, or None once the kernel
    changed or the run is not the captured configuration (the per-step sorted
    kernel at the workload's default per-cell load, leap-frog step, no cooling,
    the charge-conserving current)."""
    P = PROFILED.get(a.workload)
    default_ppc = 16 if a.workload == "beam" else 32
    if (not P or a.deposit not in ("auto", "cells") or a.ppc != default_ppc or a.integrator != 2 or a.radiation
            or a.current != "conserving" or a.filter or a.field_solver != "implicit"):
        return None
    if not PROFILED_SOURCES or any(_digest(rel) != d for rel, d in PROFILED_SOURCES.items()):
        return None
    return P


def issue_roofline(P, particle_steps, part_ms, clk):
    """Instruction issue of the particle kernel against its ceiling: the
    captured warp-instructions per particle times the particle-steps, over the
    kernel's live time, against SMs x 4 schedulers x one warp-instruction per
    cycle at the SM clock sampled during the timed region."""
    import torch
    if not P or part_ms <= 0 or not clk or not clk.get("sm_mhz"):
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    achieved = P["warp_inst_per_particle"] * particle_steps / (part_ms * 1e-3)
    peak = sms * 4 * clk["sm_mhz"] * 1e6
    return {"warp_inst_per_particle": P["warp_inst_per_particle"], "achieved": achieved, "peak": peak,
            "unit": "warp-instructions/s", "frac": achieved / peak, "sms": sms}


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["thermal", "weibel", "beam", "shock"], default="beam",
                    help="thermal / weibel: n^3 pair plasma; beam: cold Gamma=10 beam through an electron-ion "
                         "background on 2n x n x n; shock: the same beam on 2n x n x n between walls, fed "
                         "through an open end and reflected by the far wall")
    ap.add_argument("--n", type=int, default=128, help="cells per axis")
    ap.add_argument("--ppc", type=int, default=None,
                    help="macro-particles per cell per species (per population for beam); default 32, beam 16")
    ap.add_argument("--deposit", choices=["auto", "global", "tiled", "cells"], default="auto")
    ap.add_argument("--field-solver", choices=["implicit", "explicit"], default="implicit",
                    help="implicit (eq:EllipticB) or the explicit FDTD leap-frog; explicit runs at dt=0.04, "
                         "under its stability limit 0.0466 at dx=0.1")
    ap.add_argument("--current", choices=["conserving", "direct"], default="conserving",
                    help="charge-conserving high-order current, or the direct current eq:jj2")
    ap.add_argument("--filter", type=int, default=0, help="divergence-filter passes after every step (0 = off)")
    ap.add_argument("--integrator", type=int, choices=[2, 4], default=2,
                    help="2: leap-frog step; 4: four-substep 4th-order symplectic step")
    ap.add_argument("--radiation", type=float, default=0.0,
                    help="radiative-cooling coefficient mu0 q^2/(6 pi m c) for every species (0 = off)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-n", type=int, default=32, help="cells per axis of the oracle sample (the crop)")
    ap.add_argument("--sample-steps", type=int, default=2, help="steps of the oracle sample")
    ap.add_argument("--ref-sample-n", type=int, default=16,
                    help="cells per axis of the oracle sample that --impl reference times every step")
    ap.add_argument("--diag-steps", type=int, default=10,
                    help="steps after the timed region with diagnostics after each (Gauss-drift series)")
    ap.add_argument("--serve", action="store_true",
                    help="serving form: p50/p99 time-to-result of a Poisson request trace, batched vs one at a time")
    ap.add_argument("--batched", action="store_true",
                    help="batched form: 64 uneven runs advanced together against one at a time")
    ap.add_argument("--batch-steps", type=int, default=30, help="steps per run of the batched form")
    ap.add_argument("--decompose", action="store_true",
                    help="one run split over the ranks by z-slabs (parallel.py: current summed by allreduce, "
                         "particles migrate); strong scaling. Default: independent replicas, weak scaling")
    ap.add_argument("--requests", type=int, default=12)
    ap.add_argument("--rate", type=float, default=0.3, help="mean arrivals per second of the serving trace")
    ap.add_argument("--serve-scale", choices=["c5", "reduced"], default="c5")
    ap.add_argument("--serve-particles", type=int, default=48_000_000,
                    help="serving: particles the running requests may hold together before the next request "
                         "waits (0 = no limit)")
    a = ap.parse_args()
    if a.ppc is None:
        a.ppc = 16 if a.workload == "beam" else 32
    return a


def workload_grid(a, edge):
    return (2 * edge, edge, edge) if a.workload in ("beam", "shock") else (edge, edge, edge)


# open end of the shock workload: 20-cell outflow layer, particles leave 10 cells out
SHOCK_LAYER, SHOCK_DAMPING, SHOCK_ESCAPE = 20, 0.2, 10.0


def workload_dt(a):
    if a.workload in ("beam", "shock"):   # dx = 0.5; the explicit solver's limit there is 0.233
        return 0.2 if a.field_solver == "explicit" else 0.25
    return 0.04 if a.field_solver == "explicit" else 0.05


def make_load(a, edge, seed_offset=0):
    import pp_synth
    n = workload_grid(a, edge)
    if a.workload == "beam":
        L = pp_synth.beam_background(n=n, ppc=a.ppc, seed=1214 + seed_offset)
        L.dt = workload_dt(a)
        return L
    if a.workload == "shock":
        L = pp_synth.wall_beam(n=n, ppc=a.ppc, seed=1218 + seed_offset)
        L.dt = workload_dt(a)
        return L
    if a.workload == "thermal":
        return pp_synth.thermal(n=n, ppc=a.ppc, seed=1212 + seed_offset, dt=workload_dt(a))
    return pp_synth.weibel(n=n, ppc=a.ppc, seed=1213 + seed_offset, dt=workload_dt(a))


def workload_load(a, seed_offset=0):
    return make_load(a, a.n, seed_offset)


def nominal_particles(a):
    nx, ny, nz = workload_grid(a, a.n)
    return nx * ny * nz * a.ppc * 2 * (2 if a.workload == "beam" else 1)


def workload_name(a, nparticles):
    nx, ny, nz = workload_grid(a, a.n)
    if a.workload == "beam":
        head = (f"cold Gamma=10 beam through an electron-ion background (m_i/m_e=25, u_th=0.01c), "
                f"{nx}x{ny}x{nz} cells, dx=0.5, dt={workload_dt(a):g}, {a.ppc} per cell per species per population "
                f"({nparticles} particles)")
    elif a.workload == "shock":
        head = (f"wall shock: cold Gamma=10 electron-ion beam (m_i/m_e=25) between reflecting walls, "
                f"{nx}x{ny}x{nz} cells (mesh {2 * nx}x{ny}x{nz} mirror-extended), dx=0.5, dt={workload_dt(a):g}, "
                f"{a.ppc} per cell per species (about {nparticles} particles), fed through an open end at x=0 "
                f"({SHOCK_LAYER}-cell outflow layer, damping {SHOCK_DAMPING:g}, escape {SHOCK_ESCAPE:g} cells) "
                f"by a neutral Philox injector and reflected by the wall at x=L")
    else:
        kind = "thermal pair plasma u_th=0.1c (numerical heating)" if a.workload == "thermal" else \
            "Weibel counter-streaming pair beams +-0.5c, u_th=0.1c"
        head = (f"{kind}, {a.n}^3 cells, dx=0.1, dt={workload_dt(a):g}, {a.ppc} per cell per species "
                f"({nparticles} particles)")
    return (f"{head}, "
            f"PCS, 6th-order fields, alpha=0.55, Vay, sort every 20 steps, int32 cell + fp32 offset"
            + (f", radiative cooling K={a.radiation:g}" if a.radiation else "")
            + (", 4th-order symplectic step (4 kick-drift substeps)" if a.integrator == 4 else "")
            + (", explicit FDTD field solver" if a.field_solver == "explicit" else "")
            + (", direct current eq:jj2" if a.current == "direct" else "")
            + (f", {a.filter} divergence-filter passes per step" if a.filter else ""))


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x, dist, device):
    """Max of a float over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(particles_per_rank, world, steps, max_ms):
    """Whole-job throughput of independent replicas: every rank's particle-steps
    over the slowest rank's time."""
    return particles_per_rank * world * steps / (max_ms * 1e-3)


def shock_inflow_room(a, L, steps):
    """Slots the injectors of the shock workload fill in `steps` steps, per species."""
    ny, nz = L.n[1], L.n[2]
    u = L.params["u_drift"]
    rate = a.ppc * ny * nz * (u / math.sqrt(1.0 + u * u)) * L.dt / L.d[0]
    return int(math.ceil(rate * (steps + 2))) + 64


def crop_load(a, edge):
    """The workload's per-cell load on a periodic edge^3 box (the crop), or for
    the shock a (edge, edge/2, edge/2) box between walls."""
    import pp_synth
    if a.workload == "shock":
        return make_load(a, edge // 2)
    if a.workload == "beam":
        L = pp_synth.beam_background(n=(edge, edge, edge), ppc=a.ppc, seed=1214)
        L.dt = workload_dt(a)
        return L
    return make_load(a, edge)


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_sample(a, edge, steps, warmup=0, threads=1):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    same physics and per-cell loading on the crop (for the shock: a box
    between walls with its open end and injectors, the oracle's virtual images
    included in its cost).  Returns (particle-steps/s, description, seconds,
    the oracle run, its load)."""
    import oracle
    shock = a.workload == "shock"
    L = crop_load(a, edge)
    oracle.build()
    threads = oracle.set_threads(threads)
    kw = dict(field_order=6, alpha=0.55, shape_order=3, relax_tol=1e-6, relax_max_iter=200, integrator=a.integrator,
              field_solver=oracle.EXPLICIT if a.field_solver == "explicit" else oracle.IMPLICIT,
              current_mode=oracle.DIRECT if a.current == "direct" else oracle.CHARGE_CONSERVING,
              filter_passes=a.filter, filter_interval=1)
    sim = oracle.WallSimulation(L.n, L.d, L.dt, **kw) if shock else oracle.Simulation(L.n, L.d, L.dt, **kw)
    for s in L.species:
        sim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], rad=a.radiation)
    if shock:
        sim.set_open_boundary(min(SHOCK_LAYER, L.n[0] // 2), SHOCK_DAMPING, min(SHOCK_ESCAPE, L.n[0] / 4))
        for sid in range(len(L.species)):
            sim.set_injector(sid, a.ppc, (L.params["u_drift"], 0.0, 0.0), 0.0, L.params["seed"])
    if warmup:
        sim.step(warmup)
    n0 = sum(sim.counts) if shock else L.n_particles
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    nmean = (n0 + sum(sim.counts)) / 2 if shock else L.n_particles
    sample = (f"{'x'.join(str(v) for v in L.n)} cells{' between walls' if shock else ' (periodic crop)'}, "
              f"{a.ppc} per cell per species"
              f"{' per population' if a.workload == 'beam' else ''} = {L.n_particles} particles"
              f"{' at the start, about ' + str(int(nmean)) + ' over the timed steps (the oracle also steps their mirror images)' if shock else ''}, "
              f"{steps} steps, same per-cell load and parameters as the workload, C on {threads} thread(s)"
              f"{' (particle loop with per-thread current copies)' if threads > 1 else ''}")
    return nmean * steps / dt, sample, dt, sim, L, threads


def crop_error(a, pp, osim, L, steps):
    """Error of the GPU's mixed form against the FP64 oracle on the crop, after
    the same steps from the same loaded particles: per field the max
    difference over max(max|oracle|, floor), the floor being the largest
    single-species current density J_s for J and J_s t for E and B (the net
    current of a neutral beam is a small difference of large species
    currents, which FP32 rounds relative to each species' own); positions in
    cells (particles matched one to one as periodic nearest neighbours) and
    momenta relative to max|u|."""
    import numpy as np
    from scipy.spatial import cKDTree
    sim = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3, pusher=pp.PP_VAY,
                        precision=pp.PP_MIXED32, sort_interval=20, relax_max_iter=200, relax_tol=1e-6)
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]))
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    sim.step(steps)
    js = 0.0
    if a.workload == "beam":
        js = 0.5 * math.sqrt(1.0 - 1.0 / L.params["gamma_b"] ** 2)
    t = steps * L.dt
    E, B, J = sim.fields()
    out = {}
    for name, G, O, floor in (("E", E, osim.E, js * t), ("B", B, osim.B, js * t), ("J", J, osim.J, js)):
        num = max(float(np.abs(G[k] - O[k]).max()) for k in range(3))
        den = max(max(float(np.abs(O[k]).max()) for k in range(3)), floor)
        out[name] = num / den
    box = np.array([L.n[k] * L.d[k] for k in range(3)])
    dpos, du = 0.0, 0.0
    for s in range(len(L.species)):
        g, o = sim.particles(s), osim.species[s]
        P = np.stack([np.mod(g[k], box[i]) for i, k in enumerate("xyz")], 1)
        Q = np.stack([np.mod(o[k], box[i]) for i, k in enumerate("xyz")], 1)
        P = np.minimum(P, np.nextafter(box, 0))
        Q = np.minimum(Q, np.nextafter(box, 0))
        _, j = cKDTree(Q, boxsize=box).query(P, k=1)
        d = (P - Q[j] + 0.5 * box) % box - 0.5 * box
        dpos = max(dpos, float((np.abs(d) / np.asarray(L.d)).max()))
        us = max(float(np.abs(o[k]).max()) for k in ("ux", "uy", "uz"))
        du = max(du, max(float(np.abs(g[k] - o[k][j]).max()) for k in ("ux", "uy", "uz")) / us)
    diag = sim.diagnostics()
    sim.close()
    return {"steps": steps, "E": out["E"], "B": out["B"], "J": out["J"], "positions_cells": dpos,
            "momenta_rel": du, "species_current_floor": js, "gauss_drift_gpu": diag["gauss_drift_max"],
            "grid": list(L.n), "particles": L.n_particles}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, a.steps)
    rate, sample, dt, _, _, cores = oracle_sample(a, a.ref_sample_n, steps, warmup=a.warmup, threads=host_cores())
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus, "steps": steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a, nominal_particles(a)), "oracle_sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(a):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as pp

    L = workload_load(a, seed_offset=rank)
    npart = L.n_particles
    mode = {"auto": pp.PP_DEPOSIT_AUTO, "global": pp.PP_DEPOSIT_GLOBAL, "tiled": pp.PP_DEPOSIT_TILED,
            "cells": pp.PP_DEPOSIT_CELLS}[a.deposit]
    stream = torch.cuda.current_stream()

    shock = a.workload == "shock"

    def make():
        s = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3, pusher=pp.PP_VAY,
                          precision=pp.PP_MIXED32, sort_interval=20, relax_max_iter=100, relax_tol=1e-6,
                          deposit_mode=mode, stream=stream.cuda_stream,
                          boundary_x=pp.PP_BOUNDARY_WALLS if shock else pp.PP_BOUNDARY_PERIODIC)
        s.set_integrator(a.integrator)
        s.set_field_solver(pp.PP_FIELD_EXPLICIT if a.field_solver == "explicit" else pp.PP_FIELD_IMPLICIT)
        s.set_current_deposit(pp.PP_CURRENT_DIRECT if a.current == "direct" else pp.PP_CURRENT_CONSERVING)
        s.set_divergence_filter(a.filter, 1)
        return s

    # the shock's inflow: room for every step's injection, then the open end and the injectors
    extra = shock_inflow_room(a, L, a.warmup + a.steps) if shock else 0

    def open_end(s):
        if shock:
            s.set_open_boundary(SHOCK_LAYER, SHOCK_DAMPING, SHOCK_ESCAPE)
            for sid in range(len(L.species)):
                s.set_injector(sid, a.ppc, (L.params["u_drift"], 0.0, 0.0), 0.0, L.params["seed"])

    sim = make()
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]) + extra)
        sim.set_radiative_cooling(sid, a.radiation)
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    open_end(sim)
    for _ in range(a.warmup):
        sim.step(1)
    sim.sync()
    if shock:   # particles enter and leave: count the mean load of the timed steps
        n_start = sum(sim.count(sid) for sid in range(len(L.species)))

    # ---- device-resident timed region ----
    sim.profile_enable(True)
    torch.cuda.synchronize()
    barrier()
    gpu_id = getattr(torch.cuda.get_device_properties(local), "uuid", None)
    clocks = Clocks(f"GPU-{gpu_id}" if gpu_id is not None else local) if rank == 0 else None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        sim.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    barrier()
    ms = ev0.elapsed_time(ev1)
    prof = sim.profile_read()
    sim.profile_enable(False)
    sim.sync()
    if shock:
        npart = (n_start + sum(sim.count(sid) for sid in range(len(L.species)))) // 2
    ms = reduce_max(ms, dist, "cuda")
    total_particles = npart * world
    value = replica_value(npart, world, a.steps, ms)

    # roofline of the dominant kernel (the fused particle kernel)
    peak, peak_kind = measured_peak()
    part_ms = prof["particle_ms"]
    bytes_per_step = BYTES_PER_PARTICLE_STEP * (4 if a.integrator == 4 else 1)   # one particle pass per substep
    achieved = bytes_per_step * npart * a.steps / (part_ms * 1e-3) / 1e9 if part_ms > 0 else 0.0
    diag = sim.diagnostics()
    # Gauss drift after each of diag_steps further steps: max|G - G_0| with
    # G = div E - rho; a step changes G by -dt times its discrete continuity
    # residual (rho^{n+1} - rho^n)/dt + div J, so the series shows how that
    # residual adds up
    series = [diag["gauss_drift_max"]]
    for _ in range(a.diag_steps):
        sim.step(1)
        series.append(sim.diagnostics()["gauss_drift_max"])

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not a.no_e2e:
        sim.close()
        del sim
        pinned = []
        for s in L.species:
            pinned.append({k: torch.from_numpy(np.ascontiguousarray(s[k], dtype=np.float64)).pin_memory()
                           for k in ("x", "y", "z", "ux", "uy", "uz")})
        h2d = sum(sum(t.numel() * 8 for t in p.values()) for p in pinned)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        sim2 = make()
        for s, p in zip(L.species, pinned):
            sid = sim2.add_species(s["q"], s["m"], s["w"], len(s["x"]) + extra)
            sim2.set_radiative_cooling(sid, a.radiation)
            sim2.load_particles(sid, *[p[k].numpy() for k in ("x", "y", "z", "ux", "uy", "uz")])
        open_end(sim2)
        sim2.step(a.steps)
        d2 = sim2.diagnostics()
        t1 = time.perf_counter()
        el = reduce_max(t1 - t0, dist, "cuda")
        e2e = {"value": total_particles * a.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": h2d // max(1, a.steps), "d2h_bytes_per_step": 200 // max(1, a.steps),
               "seconds": el, "status": d2["status"]}
        sim2.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu, crop = None, None
    if not a.no_cpu_baseline:
        rate, sample, _, osim, Lc, cores = oracle_sample(a, a.sample_n, steps=a.sample_steps, threads=host_cores())
        rate1, sample1, _, _, _, _ = oracle_sample(a, a.sample_n, steps=1, threads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1, "sample": sample1}}
        if a.workload != "shock":   # the crop's error: the GPU's mixed form on the oracle's sample
            crop = crop_error(a, pp, osim, Lc, a.sample_steps)
    P = profiled(a)
    per_launch = npart * a.steps / max(1, prof["particle_launches"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a, npart), "grid": list(workload_grid(a, a.n)), "particles_per_gpu": npart,
                   "precision": "mixed (int32 cell + fp32 offset; fp32 fields and current; fp64 reductions)",
                   "deposit": a.deposit, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (particle state 28 B x particles, read and written every step)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": P["bytes_per_particle"] * per_launch if P else None,
                     "limiter": P["limiter"] if P else None, "issue": issue_roofline(P, npart * a.steps, part_ms, clk),
                     "kernel": "fused particle step (gather+push+move+deposit)",
                     "bytes_per_particle_step": bytes_per_step, "peak_kind": peak_kind,
                     "kernel_ms_per_step": part_ms / a.steps},
        "cpu_baseline": cpu,
        "oracle_error": crop,
        "e2e": e2e,
        "gpu_launches": prof["kernel_launches"],
        "clocks": clk,
        "phases_ms_per_step": {k: prof[k] / a.steps for k in ("particle_ms", "current_ms", "field_ms", "sort_ms")},
        "diag": {"status": diag["status"], "gauss_drift_rel": diag["gauss_drift_max"] / max(diag["rho_max"], 1e-300),
                 "gauss_drift_max": diag["gauss_drift_max"], "rho_max": diag["rho_max"],
                 # every workload loads a charge density of 1 per sign (electrons: -1)
                 "gauss_drift_vs_species_density": diag["gauss_drift_max"],
                 "relax_residual": diag["relax_residual"], "relax_iters": diag["relax_iters"],
                 "gauss_drift_series_vs_species_density": series,
                 "gauss_drift_growth_per_step_max": max((abs(b - c) for b, c in zip(series[1:], series[:-1])),
                                                        default=0.0)},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serve(a):
    """Serving form: a Poisson trace of independent two-stream / Weibel runs
    served by continuous batching through pp_batch_* (admission by device
    bytes and by a particle budget, every run resident, steps overlapping on
    the GPU), against the same requests run one at a time.  Default trace: the
    serving configuration's distributions (edges 32..192, 8..32 ppc per
    species, pair or m_i/m_e = 25, 200..1000 steps) at 0.3 arrivals/s, which
    the GPU just saturates; `--serve-scale reduced` takes edges 16..48 and
    20..100 steps instead."""
    import pp_synth
    from paper_1211_4575_gb300 import build
    build.build()
    from paper_1211_4575_gb300 import serving
    if a.serve_scale == "c5":
        edges, steps, desc = tuple(range(32, 193, 16)), (200, 1000), "edges 32..192, 200..1000 steps"
        budget, slots = 200 << 30, 8
    else:
        edges, steps, desc = (16, 24, 32, 40, 48), (20, 100), "edges 16..48, 20..100 steps"
        budget, slots = 64 << 30, 32
    trace = pp_synth.serving_trace(n_requests=a.requests, rate=a.rate, edges=edges, steps=steps)
    warm = [dict(r, arrival=0.0, steps=2, n=32) for r in trace[:2]]
    serving.sequential(warm)
    seq, _ = serving.sequential(trace)
    bat, _ = serving.serve(trace, budget_bytes=budget, max_slots=slots, chunk=4,
                           max_active_particles=a.serve_particles or None)
    work = sum(r["n"] ** 3 * max(2, r["ppc"] // 2 * 2) * 2 * r["steps"] for r in trace)
    line = {"metric": "serving p50/p99 time-to-result", "value": bat["p99_s"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{a.requests} Poisson arrivals at {a.rate}/s of two-stream/Weibel runs, "
                                   f"{desc}, 8..32 ppc per species, pair or m_i/m_e=25, mixed precision, PCS; "
                                   f"budget {budget >> 30} GiB, {slots} slots, "
                                   f"particle budget {a.serve_particles or 'none'}; loads built by 4 host worker threads "
                                   "in both forms; time to result from arrival to the end of the last step",
                       "offered_particle_steps": work},
            "batched": bat, "sequential": seq}
    print(json.dumps(line), flush=True)


def run_batched(a):
    """Batched form: the 64 runs of uneven size of the batched config (edges
    16..96, 8..64 ppc, TSC or PCS, mixed precision) with `--batch-steps` steps
    each instead of 300, loads resident before the clock starts; all runs in
    slots on their own streams (graph-captured steps, and without graphs)
    against the same runs one at a time.  The loads are built once; each leg
    continues the runs where the previous one left them."""
    import pp_synth
    from paper_1211_4575_gb300 import build
    build.build()
    from paper_1211_4575_gb300 import serving
    runs = pp_synth.batched_runs(steps=a.batch_steps)
    built = serving.build_all(runs)
    serving.one_at_a_time([(dict(r, steps=1),) + tuple(b[1:]) for r, b in zip(runs[:2], built[:2])])   # warm-up
    seq = serving.one_at_a_time(built)
    eager = serving.batched(built, budget_bytes=160 << 30, max_slots=64, chunk=4, graphs=False)
    bat = serving.batched(built, budget_bytes=160 << 30, max_slots=64, chunk=4, graphs=True)
    fused = serving.batched(built, budget_bytes=160 << 30, max_slots=64, chunk=4, graphs=False, fused=True)
    for _, sim, _, _ in built:
        sim.close()
    best = max((fused, bat, eager), key=lambda r: r["particle_steps_per_s"])
    line = {"metric": "particle-steps/s (gather+push+deposit)", "value": best["particle_steps_per_s"],
            "unit": "particle-steps/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"64 independent two-stream pair runs, edges 16..96, 8..64 ppc per species, "
                                   f"drift 0.05..0.5c, u_th 0.01..0.1c, TSC or PCS, {a.batch_steps} steps each, "
                                   "mixed precision, loads resident before timing; 64 slots, one stream each"},
            "batched_fused": fused, "batched_graphs": bat, "batched_eager": eager, "one_at_a_time": seq}
    print(json.dumps(line), flush=True)


def run_decomposed(a):
    """One run of the workload split over the ranks by z-slabs: every rank
    holds the mesh and the particles of its slab; per step the particle pass,
    the allreduce of the current (NCCL), the field update and the migration of
    the particles that changed slab (paper_1211_4575_gb300.parallel)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29533")
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local))
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as pp
    from paper_1211_4575_gb300 import parallel
    if a.workload not in ("thermal", "weibel", "beam"):
        raise SystemExit("--decompose runs the periodic workloads")
    L = workload_load(a)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    bounds = parallel.slab_bounds(L.n[2], L.d[2], world)
    sim = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=3, pusher=pp.PP_VAY,
                        precision=pp.PP_MIXED32, sort_interval=20, relax_max_iter=100, relax_tol=1e-6,
                        stream=stream.cuda_stream)
    for s in L.species:   # room for the particles that migrate in
        sim.add_species(s["q"], s["m"], s["w"], int(1.5 * len(s["x"]) / world) + 4096)
    sl = parallel.Slab(sim, rank, bounds, len(L.species))
    parallel.load([sl], L.species)
    comm = parallel.TorchComm(device=dev)
    for _ in range(a.warmup):
        parallel.step([sl], comm, device=dev)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        parallel.step([sl], comm, device=dev)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = reduce_max(ev0.elapsed_time(ev1), dist, "cuda")
    wall = reduce_max(time.perf_counter() - t0, dist, "cuda")
    kin, count = parallel.kinetic_and_count([sl], comm)
    if rank == 0:
        line = {"metric": METRIC, "value": L.n_particles * a.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(a, L.n_particles), "grid": list(L.n),
                           "parallelism": f"z-slabs x{world} (current allreduce, particle migration, "
                                          "replicated field update)"},
                "wall_s": wall, "particles_after": count}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    a = args()
    if a.impl == "reference":
        run_reference(a)
    elif a.decompose:
        run_decomposed(a)
    elif a.batched:
        run_batched(a)
    elif a.serve:
        run_serve(a)
    else:
        run_gpu(a)
