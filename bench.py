#!/usr/bin/env python
"""Throughput benchmark of the GB300 Photon-Plasma particle step.

One "step" is one full leap-frog step of the library (pp_step): per species the
fused gather -> push -> move -> charge-conserving deposit kernel, ghost fold,
6th-order current solve, implicit field update, and the cell sort every 20
steps.  Workload (default): the numerical-heating plasma of the paper's
Sec. VIII scaled to 3D, 128^3 cells, 32 macro-particles per cell per species
(134,217,728 particles), PCS shapes, 6th-order fields, mixed precision (int32
cell + FP32 offset).  Inputs are seeded synthetic loads (pp_synth).

Prints one JSON line (rank 0).  Multi-GPU: every rank advances its own
independent plasma (replicas, weak scaling); no collective on the data path.
`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of
the same workload.
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

# DRAM traffic of the fused particle kernel per particle, from the committed ncu
# capture of the 64^3 x 32 ppc thermal workload kept under profiles/ (traffic
# grows with the particle count).  Valid only for the kernel sources it was
# taken on: the device part of the header (up to its host-side context), the
# sort (its key sets the particle order the kernel streams) and the part of
# pp_particles.cu that holds the particle kernels (up to its charge-density
# section).
PROFILED_BYTES_PER_PARTICLE = 901.598720e6 / 16777216
# The same capture's issue and shared-memory figures, reported beside the HBM
# fraction (the kernel is bound by shared-memory issue, not by DRAM).
PROFILED_ISSUE = {"issue_active_pct": 57.0, "warp_instructions_per_particle": 111.4,
                  "shared_wavefronts_per_particle": {"load": 14.0, "atomic": 12.8},
                  "shared_bank_conflicts_per_particle": {"load": 0.5, "atomic": 6.4},
                  "top_stall": "mio_throttle (shared-memory pipe)",
                  "source": "profiles/k_particles_tiled_thermal64.md"}
_KERNEL_END = "// ---------------------------------------------------------------------------\n// Charge density of eq:rho2"
_HOST_START = "// ---------------------------------------------------------------------------\n// Context (host side)"
PROFILED_SOURCES = {
    "paper_1211_4575_gb300/csrc/pp_particles.cu": "3285fa49a9cf12f024223f16ec4ccb565f4802fa407807e82e696a22d8cd2b5d",
    "paper_1211_4575_gb300/csrc/pp_internal.cuh": "643a48f3cec37d301be2db1853792dc3ef6c269944bb793e18bc1b1ae96f6b0b",
    "paper_1211_4575_gb300/csrc/pp_sort.cu": "8ae278e854810bdf3db42a7069642a62f7c7a0c1cddf9bd8d09dca831784555a",
}


def profiled_matches():
    """True while the particle-kernel sources are the ones the committed capture was taken on."""
    import hashlib
    for rel, digest in PROFILED_SOURCES.items():
        with open(os.path.join(ROOT, rel)) as f:
            text = f.read()
        if rel.endswith("pp_particles.cu"):
            text = text[: text.index(_KERNEL_END)]
        elif rel.endswith("pp_internal.cuh"):
            text = text[: text.index(_HOST_START)]
        if hashlib.sha256(text.encode()).hexdigest() != digest:
            return False
    return True


def profiled_traffic(particles_per_launch):
    """ncu DRAM bytes per launch scaled to this launch, or None once the kernel changed."""
    return PROFILED_BYTES_PER_PARTICLE * particles_per_launch if profiled_matches() else None


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["thermal", "weibel", "beam", "shock"], default="thermal",
                    help="thermal / weibel: n^3 pair plasma; beam: cold Gamma=10 beam through an electron-ion "
                         "background on 2n x n x n; shock: the same beam on 2n x n x n between walls, fed "
                         "through an open end and reflected by the far wall")
    ap.add_argument("--n", type=int, default=128, help="cells per axis")
    ap.add_argument("--ppc", type=int, default=None,
                    help="macro-particles per cell per species (per population for beam); default 32, beam 16")
    ap.add_argument("--deposit", choices=["auto", "global", "tiled"], default="auto")
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
    ap.add_argument("--sample-n", type=int, default=16, help="cells per axis of the oracle sample")
    ap.add_argument("--serve", action="store_true",
                    help="serving form: p50/p99 time-to-result of a Poisson request trace, batched vs one at a time")
    ap.add_argument("--batched", action="store_true",
                    help="batched form: 64 uneven runs advanced together against one at a time")
    ap.add_argument("--batch-steps", type=int, default=30, help="steps per run of the batched form")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=20.0)
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


def oracle_rate(a, steps, warmup=0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    same physics and per-cell loading on a sample_n^3 periodic box (for the
    shock: a (sample_n, sample_n/2, sample_n/2) box between walls with its open
    end and injectors, the oracle's virtual images included in its cost)."""
    import oracle
    import pp_synth
    shock = a.workload == "shock"
    L = make_load(a, a.sample_n // 2 if shock else a.sample_n)
    oracle.build()
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
    nmean = (n0 + sum(sim.counts)) / 2 if shock else L.n_particles
    sample = (f"{'x'.join(str(v) for v in L.n)} cells{' between walls' if shock else ''}, "
              f"{a.ppc} per cell per species"
              f"{' per population' if a.workload == 'beam' else ''} = {L.n_particles} particles"
              f"{' at the start, about ' + str(int(nmean)) + ' over the timed steps (the oracle also steps their mirror images)' if shock else ''}, "
              f"{steps} steps, same per-cell load and parameters as the workload, single-threaded C")
    return nmean * steps / dt, sample, dt


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, a.steps)
    rate, sample, dt = oracle_rate(a, steps, warmup=a.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus, "steps": steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a, nominal_particles(a)), "oracle_sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    mode = {"auto": pp.PP_DEPOSIT_AUTO, "global": pp.PP_DEPOSIT_GLOBAL, "tiled": pp.PP_DEPOSIT_TILED}[a.deposit]
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
    cpu = None
    if not a.no_cpu_baseline:
        rate, sample, _ = oracle_rate(a, steps=5)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
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
                     "traffic": profiled_traffic(npart * a.steps / max(1, prof["particle_launches"])),
                     "issue": PROFILED_ISSUE if profiled_matches() else None,
                     "kernel": "fused particle step (gather+push+move+deposit)",
                     "bytes_per_particle_step": bytes_per_step, "peak_kind": peak_kind,
                     "kernel_ms_per_step": part_ms / a.steps},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": prof["kernel_launches"],
        "clocks": clk,
        "phases_ms_per_step": {k: prof[k] / a.steps for k in ("particle_ms", "current_ms", "field_ms", "sort_ms")},
        "diag": {"status": diag["status"], "gauss_drift_rel": diag["gauss_drift_max"] / max(diag["rho_max"], 1e-300),
                 "gauss_drift_max": diag["gauss_drift_max"], "rho_max": diag["rho_max"],
                 # every workload loads a charge density of 1 per sign (electrons: -1)
                 "gauss_drift_vs_species_density": diag["gauss_drift_max"],
                 "relax_residual": diag["relax_residual"], "relax_iters": diag["relax_iters"]},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serve(a):
    """Serving form on a reduced Poisson trace (same distributions as the
    serving config, edges 16..48 and 20..100 steps so that it ends in minutes):
    continuous batching through pp_batch_* against the same requests run one
    at a time."""
    import torch
    import pp_synth
    from paper_1211_4575_gb300 import build
    build.build()
    from paper_1211_4575_gb300 import serving
    trace = pp_synth.serving_trace(n_requests=a.requests, rate=a.rate, edges=(16, 24, 32, 40, 48), steps=(20, 100))
    warm = [dict(r, arrival=0.0, steps=2) for r in trace[:2]]
    serving.sequential(warm)
    seq, _ = serving.sequential(trace)
    bat, _ = serving.serve(trace, budget_bytes=64 << 30, max_slots=32, chunk=4)
    line = {"metric": "serving p50/p99 time-to-result", "value": bat["p99_s"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{a.requests} Poisson arrivals at {a.rate}/s of two-stream/Weibel runs, "
                                   "edges 16..48, 8..32 ppc per species, pair or m_i/m_e=25, 20..100 steps, "
                                   "mixed precision, PCS; budget 64 GiB, 32 slots"},
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
    for _, sim, _, _ in built:
        sim.close()
    line = {"metric": "particle-steps/s (gather+push+deposit)", "value": bat["particle_steps_per_s"],
            "unit": "particle-steps/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"64 independent two-stream pair runs, edges 16..96, 8..64 ppc per species, "
                                   f"drift 0.05..0.5c, u_th 0.01..0.1c, TSC or PCS, {a.batch_steps} steps each, "
                                   "mixed precision, loads resident before timing; 64 slots, one stream each"},
            "batched_graphs": bat, "batched_eager": eager, "one_at_a_time": seq}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = args()
    if a.impl == "reference":
        run_reference(a)
    elif a.batched:
        run_batched(a)
    elif a.serve:
        run_serve(a)
    else:
        run_gpu(a)
